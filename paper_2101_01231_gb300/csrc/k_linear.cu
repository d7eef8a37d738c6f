// FP64 kernels of the linear-flux RIDG step.
//
// Prediction (Sec. 2.2): for a linear flux on a uniform periodic mesh the region system
// of eq. pred_full_system is the same for every cell, so the kept centre coefficients
// are W_i = P X_i with X_i the theta_S coefficients of the region cells upstream of cell i
// (the upwind box, 2^d of the 3^d cells for a velocity with no zero component; the others
// have zero columns) gathered with periodic wrap, and P the centre rows of the region
// solution operator.
//
// Correction (Sec. 2.3): with W-bar the time mean of W (all a linear flux needs, since
// int psi_g dtau = 2 delta_g0),
//   dQ_i = sum_d nu_d (D along d) Wbar_i
//          - sum_d [ phi(+1) (x)_d F_{i+1/2} - phi(-1) (x)_d F_{i-1/2} ],
//   F_{i+1/2} = nu+_d trace_{+1}(Wbar_i) + nu-_d trace_{-1}(Wbar_{i+e_d}).
// Each face value is evaluated by one device function with a fixed fma order from the
// same inputs on both sides of the face, so the two neighbours apply bitwise the same
// flux and the cell averages are conserved to round-off of the final additions.
#include <cuda_runtime.h>

#include "ridg_internal.h"

namespace ridg {
namespace {

constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

struct Coords {
  int x, y, z;
};

// (cell counts stay below 2^31: 32-bit division, far cheaper than 64-bit)
__device__ __forceinline__ Coords cell_coords(long long e, int nx, int ny) {
  Coords c;
  const unsigned u = (unsigned)e, r = u / (unsigned)nx;
  c.x = (int)(u - r * (unsigned)nx);
  c.y = (int)(r % (unsigned)ny);
  c.z = (int)(r / (unsigned)ny);
  return c;
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <int DIM>
__device__ __forceinline__ long long neighbour(const Coords& c, int ox, int oy, int oz, int nx,
                                               int ny, int nz) {
  long long j = wrap(c.x + ox, nx);
  if (DIM > 1) j += (long long)nx * wrap(c.y + oy, ny);
  if (DIM > 2) j += (long long)nx * ny * wrap(c.z + oz, nz);
  return j;
}

// ---------------------------------------------------------------------------------------
// prediction: each thread owns one cell and CH consecutive output rows of P
// ---------------------------------------------------------------------------------------
template <int DIM, int NB, int CH>
__global__ void __launch_bounds__(128) predict_fp64_kernel(const double* __restrict__ Q,
                                                           const double* __restrict__ P, int nout,
                                                           double* __restrict__ W, int wstride,
                                                           int nx, int ny, int nz, long long ncell,
                                                           RegionBox box) {
  constexpr int THS = ipow_c(NB, DIM);
  const int K = box.n * THS;
  extern __shared__ double sP[];  // CH x K
  const int c0 = blockIdx.y * CH;
  for (int i = threadIdx.x; i < CH * K; i += blockDim.x) {
    const int c = c0 + i / K;
    sP[i] = (c < nout) ? P[(size_t)c * K + (i % K)] : 0.0;
  }
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const Coords c = cell_coords(e, nx, ny);
  double acc[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) acc[j] = 0.0;
#pragma unroll 1
  for (int r = 0; r < box.n; ++r) {
    const int ox = box.lo[0] + r % box.cnt[0];
    const int oy = box.lo[1] + (r / box.cnt[0]) % box.cnt[1];
    const int oz = box.lo[2] + r / (box.cnt[0] * box.cnt[1]);
    const double* q = Q + neighbour<DIM>(c, ox, oy, oz, nx, ny, nz) * THS;
    const double* p = sP + r * THS;
#pragma unroll
    for (int s = 0; s < THS; ++s) {
      const double x = __ldg(q + s);
#pragma unroll
      for (int j = 0; j < CH; ++j) acc[j] = fma(p[j * K + s], x, acc[j]);
    }
  }
  double* w = W + e * wstride + c0;
#pragma unroll
  for (int j = 0; j < CH; ++j)
    if (c0 + j < nout) w[j] = acc[j];
}

// ---------------------------------------------------------------------------------------
// correction
// ---------------------------------------------------------------------------------------
// trace of a cell's time mean along dimension dd: tr[t] = sum_b v[b] w[base(t) + b st]
template <int DIM, int NB>
__device__ __forceinline__ void face_trace(const double* w, int dd, const double* v,
                                           double* tr) {
  constexpr int NT = ipow_c(NB, DIM - 1);
  const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int lo = t % st, hi = t / st;
    const int base = lo + hi * st * NB;
    double a = 0.0;
#pragma unroll
    for (int b = 0; b < NB; ++b) a = fma(v[b], w[base + b * st], a);
    tr[t] = a;
  }
}

// The single definition of a face value from the two traces at that face (explicit fma,
// so both neighbours evaluate it bit-identically).
__device__ __forceinline__ double face_value(double tr_left_plus, double tr_right_minus, double nup,
                                          double num) {
  return fma(nup, tr_left_plus, num * tr_right_minus);
}

template <int DIM, int NB>
__global__ void __launch_bounds__(128) correct_linear_kernel(double* __restrict__ Q,
                                                             const double* __restrict__ Wb,
                                                             int wstride, int nx, int ny, int nz,
                                                             long long ncell, CorrParams cp) {
  constexpr int THS = ipow_c(NB, DIM);
  constexpr int NT = ipow_c(NB, DIM - 1);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const Coords c = cell_coords(e, nx, ny);
  double w[THS], dq[THS], nbw[THS];
#pragma unroll
  for (int s = 0; s < THS; ++s) {
    w[s] = Wb[e * wstride + s];
    dq[s] = 0.0;
  }
#pragma unroll
  for (int dd = 0; dd < DIM; ++dd) {
    const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
    // volume term nu_d (D along d) Wbar
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int base = t % st + (t / st) * st * NB;
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (a > b && ((a + b) & 1)) acc = fma(cp.D[a * kMaxNB + b], w[base + b * st], acc);
        dq[base + a * st] = fma(cp.nu[dd], acc, dq[base + a * st]);
      }
    }
    double trp[NT], trm[NT], nbt[NT], fp[NT], fm[NT];
    face_trace<DIM, NB>(w, dd, cp.ep, trp);
    face_trace<DIM, NB>(w, dd, cp.em, trm);
    // right neighbour's trace at its xi_d = -1
    {
      const long long j = neighbour<DIM>(c, dd == 0, dd == 1, dd == 2, nx, ny, nz);
#pragma unroll
      for (int s = 0; s < THS; ++s) nbw[s] = Wb[j * wstride + s];
      face_trace<DIM, NB>(nbw, dd, cp.em, nbt);
#pragma unroll
      for (int t = 0; t < NT; ++t) fp[t] = face_value(trp[t], nbt[t], cp.nup[dd], cp.num[dd]);
    }
    // left neighbour's trace at its xi_d = +1
    {
      const long long j = neighbour<DIM>(c, -(dd == 0), -(dd == 1), -(dd == 2), nx, ny, nz);
#pragma unroll
      for (int s = 0; s < THS; ++s) nbw[s] = Wb[j * wstride + s];
      face_trace<DIM, NB>(nbw, dd, cp.ep, nbt);
#pragma unroll
      for (int t = 0; t < NT; ++t) fm[t] = face_value(nbt[t], trm[t], cp.nup[dd], cp.num[dd]);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int base = t % st + (t / st) * st * NB;
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        double v = dq[base + a * st];
        v = fma(-cp.ep[a], fp[t], v);
        v = fma(cp.em[a], fm[t], v);
        dq[base + a * st] = v;
      }
    }
  }
  double* q = Q + e * THS;
#pragma unroll
  for (int s = 0; s < THS; ++s) q[s] = q[s] + dq[s];
}

// The same correction with one thread per (cell, mode) output, for large theta_S (3D,
// degree >= 4) where a thread holding a whole cell's time mean would spill.  Mode s has the
// digit a = s_d along dimension d and lies on the fibre base + b st of that dimension; every
// sum runs in the order of correct_linear_kernel (volume term, then the two face values,
// each face value from the same traces by face_value), so both neighbours of a face apply
// bitwise the same flux and the result equals correct_linear_kernel's bit for bit.
template <int DIM, int NB>
__global__ void __launch_bounds__(128) correct_modes_kernel(double* __restrict__ Q,
                                                            const double* __restrict__ Wb,
                                                            int wstride, int nx, int ny, int nz,
                                                            long long ncell, CorrParams cp) {
  constexpr int THS = ipow_c(NB, DIM);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell * THS) return;
  const long long e = i / THS;
  const int s = (int)(i - e * THS);
  const Coords c = cell_coords(e, nx, ny);
  const double* w = Wb + e * wstride;
  double dq = 0.0;
#pragma unroll
  for (int dd = 0; dd < DIM; ++dd) {
    const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
    const int a = (s / st) % NB, base = s - a * st;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < a && ((a + b) & 1)) acc = fma(cp.D[a * kMaxNB + b], w[base + b * st], acc);
    dq = fma(cp.nu[dd], acc, dq);
    double trp = 0.0, trm = 0.0, nbp = 0.0, nbm = 0.0;
    const double* wr = Wb + neighbour<DIM>(c, dd == 0, dd == 1, dd == 2, nx, ny, nz) * wstride;
    const double* wl = Wb + neighbour<DIM>(c, -(dd == 0), -(dd == 1), -(dd == 2), nx, ny, nz) * wstride;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      trp = fma(cp.ep[b], w[base + b * st], trp);
      trm = fma(cp.em[b], w[base + b * st], trm);
      nbm = fma(cp.em[b], wr[base + b * st], nbm);
      nbp = fma(cp.ep[b], wl[base + b * st], nbp);
    }
    const double fp = face_value(trp, nbm, cp.nup[dd], cp.num[dd]);
    const double fm = face_value(nbp, trm, cp.nup[dd], cp.num[dd]);
    dq = fma(-cp.ep[a], fp, dq);
    dq = fma(cp.em[a], fm, dq);
  }
  Q[e * THS + s] = Q[e * THS + s] + dq;
}

// A whole run of n steps of a small 1D mesh in one CTA: the state and the time means stay in
// shared memory, each step is the prediction (the same sums as predict_fp64_kernel) and the
// correction (the same sums as correct_linear_kernel<1, NB>) separated by barriers.  Removes
// the two launches per step that bound tiny meshes.
template <int NB>
__global__ void __launch_bounds__(256) run1d_fp64_kernel(double* __restrict__ Q,
                                                         const double* __restrict__ P, int n,
                                                         int nsteps, CorrParams cp, int lo, int nr) {
  const int K = nr * NB;     // the upwind cells lo .. lo + nr - 1 of the region
  extern __shared__ double sm1[];
  double* sP = sm1;          // NB x K (the time-mean rows)
  double* sQ = sP + NB * K;  // n x NB
  double* sW = sQ + n * NB;  // n x NB
  for (int i = threadIdx.x; i < NB * K; i += blockDim.x) sP[i] = P[i];
  for (int i = threadIdx.x; i < n * NB; i += blockDim.x) sQ[i] = Q[i];
  __syncthreads();
  for (int step = 0; step < nsteps; ++step) {
    for (int i = threadIdx.x; i < n * NB; i += blockDim.x) {
      const int c = i / NB, k = i % NB;
      double acc = 0.0;
      for (int r = 0; r < nr; ++r) {
        const double* q = sQ + wrap(c + lo + r, n) * NB;
        const double* p = sP + k * K + r * NB;
#pragma unroll
        for (int s2 = 0; s2 < NB; ++s2) acc = fma(p[s2], q[s2], acc);
      }
      sW[i] = acc;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const double* w = sW + c * NB;
      double dq[NB];
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (a > b && ((a + b) & 1)) acc = fma(cp.D[a * kMaxNB + b], w[b], acc);
        dq[a] = fma(cp.nu[0], acc, 0.0);
      }
      double trp, trm, nbt;
      face_trace<1, NB>(w, 0, cp.ep, &trp);
      face_trace<1, NB>(w, 0, cp.em, &trm);
      face_trace<1, NB>(sW + wrap(c + 1, n) * NB, 0, cp.em, &nbt);
      const double fp = face_value(trp, nbt, cp.nup[0], cp.num[0]);
      face_trace<1, NB>(sW + wrap(c - 1, n) * NB, 0, cp.ep, &nbt);
      const double fm = face_value(nbt, trm, cp.nup[0], cp.num[0]);
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        double v = dq[a];
        v = fma(-cp.ep[a], fp, v);
        v = fma(cp.em[a], fm, v);
        sQ[c * NB + a] = sQ[c * NB + a] + v;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n * NB; i += blockDim.x) Q[i] = sQ[i];
}

template <int NB>
cudaError_t run1d_dispatch(const Grid& g, double* Q, const double* P, int nsteps,
                           const CorrParams& cp, cudaStream_t s) {
  const size_t smem = (size_t)(NB * g.box.n * NB + 2 * g.ncell * NB) * sizeof(double);
  auto kern = run1d_fp64_kernel<NB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<1, 256, smem, s>>>(Q, P, (int)g.ncell, nsteps, cp, g.box.lo[0], g.box.cnt[0]);
  return cudaGetLastError();
}

template <int DIM, int NB>
cudaError_t predict_dispatch_ch(const Grid& g, const double* Q, const double* P, int nout,
                                double* W, int wstride, cudaStream_t s) {
  constexpr int THS = ipow_c(NB, DIM);
  constexpr int KMAX = ipow_c(2, DIM) * THS;  // the largest upwind box: 2^d cells
  // rows per thread: as many as fit 48 KB of shared memory, at most 16
  constexpr int CH = (16 * KMAX * 8 <= 48 * 1024) ? 16 : ((8 * KMAX * 8 <= 48 * 1024) ? 8 : 4);
  if (g.box.n < 1 || g.box.n > ipow_c(2, DIM)) return cudaErrorInvalidValue;
  const int K = g.box.n * THS;
  const int threads = 128;
  dim3 grid((unsigned)((g.ncell + threads - 1) / threads), (unsigned)((nout + CH - 1) / CH));
  size_t smem = (size_t)CH * K * sizeof(double);
  auto kern = predict_fp64_kernel<DIM, NB, CH>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, threads, smem, s>>>(Q, P, nout, W, wstride, g.n[0], g.n[1], g.n[2], g.ncell, g.box);
  return cudaGetLastError();
}

template <int DIM, int NB>
cudaError_t correct_dispatch(const Grid& g, double* Q, const double* Wb, int wstride,
                             const CorrParams& cp, cudaStream_t s) {
  const int threads = 128;
  if constexpr (DIM == 3 && NB >= 5) {
    const unsigned blocks = (unsigned)((g.ncell * ipow_c(NB, DIM) + threads - 1) / threads);
    correct_modes_kernel<DIM, NB><<<blocks, threads, 0, s>>>(Q, Wb, wstride, g.n[0], g.n[1],
                                                             g.n[2], g.ncell, cp);
  } else {
    const unsigned blocks = (unsigned)((g.ncell + threads - 1) / threads);
    correct_linear_kernel<DIM, NB><<<blocks, threads, 0, s>>>(Q, Wb, wstride, g.n[0], g.n[1],
                                                              g.n[2], g.ncell, cp);
  }
  return cudaGetLastError();
}

}  // namespace

#define RIDG_DISPATCH_NB(DIM, FN, ...)                 \
  switch (nb) {                                        \
    case 1: return FN<DIM, 1>(__VA_ARGS__);            \
    case 2: return FN<DIM, 2>(__VA_ARGS__);            \
    case 3: return FN<DIM, 3>(__VA_ARGS__);            \
    case 4: return FN<DIM, 4>(__VA_ARGS__);            \
    default: break;                                    \
  }

cudaError_t launch_predict_fp64(const Grid& g, int nb, const double* Q, const double* P, int nout,
                                double* W, int wstride, cudaStream_t s) {
  if (g.dim == 1) {
    RIDG_DISPATCH_NB(1, predict_dispatch_ch, g, Q, P, nout, W, wstride, s)
    switch (nb) {
      case 5: return predict_dispatch_ch<1, 5>(g, Q, P, nout, W, wstride, s);
      case 6: return predict_dispatch_ch<1, 6>(g, Q, P, nout, W, wstride, s);
      case 7: return predict_dispatch_ch<1, 7>(g, Q, P, nout, W, wstride, s);
      case 8: return predict_dispatch_ch<1, 8>(g, Q, P, nout, W, wstride, s);
      case 9: return predict_dispatch_ch<1, 9>(g, Q, P, nout, W, wstride, s);
      case 10: return predict_dispatch_ch<1, 10>(g, Q, P, nout, W, wstride, s);
      case 11: return predict_dispatch_ch<1, 11>(g, Q, P, nout, W, wstride, s);
      case 12: return predict_dispatch_ch<1, 12>(g, Q, P, nout, W, wstride, s);
      default: break;
    }
  } else if (g.dim == 2) {
    RIDG_DISPATCH_NB(2, predict_dispatch_ch, g, Q, P, nout, W, wstride, s)
    switch (nb) {
      case 5: return predict_dispatch_ch<2, 5>(g, Q, P, nout, W, wstride, s);
      case 6: return predict_dispatch_ch<2, 6>(g, Q, P, nout, W, wstride, s);
      default: break;
    }
  } else if (g.dim == 3) {
    RIDG_DISPATCH_NB(3, predict_dispatch_ch, g, Q, P, nout, W, wstride, s)
    switch (nb) {
      case 5: return predict_dispatch_ch<3, 5>(g, Q, P, nout, W, wstride, s);
      case 6: return predict_dispatch_ch<3, 6>(g, Q, P, nout, W, wstride, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

bool run1d_fits(const Grid& g, int nb) {
  return g.dim == 1 && nb >= 1 && nb <= kMaxNB && g.ncell <= kRun1dMaxCells &&
         g.box.n >= 1 && g.box.n <= 2 &&
         (size_t)(g.box.n * nb * nb + 2 * g.ncell * nb) * sizeof(double) <= 96 * 1024;
}

cudaError_t launch_run1d_fp64(const Grid& g, int nb, double* Q, const double* P, int nsteps,
                              const CorrParams& cp, cudaStream_t s) {
  if (!run1d_fits(g, nb)) return cudaErrorInvalidValue;
  switch (nb) {
    case 1: return run1d_dispatch<1>(g, Q, P, nsteps, cp, s);
    case 2: return run1d_dispatch<2>(g, Q, P, nsteps, cp, s);
    case 3: return run1d_dispatch<3>(g, Q, P, nsteps, cp, s);
    case 4: return run1d_dispatch<4>(g, Q, P, nsteps, cp, s);
    case 5: return run1d_dispatch<5>(g, Q, P, nsteps, cp, s);
    case 6: return run1d_dispatch<6>(g, Q, P, nsteps, cp, s);
    case 7: return run1d_dispatch<7>(g, Q, P, nsteps, cp, s);
    case 8: return run1d_dispatch<8>(g, Q, P, nsteps, cp, s);
    case 9: return run1d_dispatch<9>(g, Q, P, nsteps, cp, s);
    case 10: return run1d_dispatch<10>(g, Q, P, nsteps, cp, s);
    case 11: return run1d_dispatch<11>(g, Q, P, nsteps, cp, s);
    case 12: return run1d_dispatch<12>(g, Q, P, nsteps, cp, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_correct_linear(const Grid& g, int nb, double* Q, const double* Wbar,
                                  int wstride, const CorrParams& cp, cudaStream_t s) {
  if (g.dim == 1) {
    RIDG_DISPATCH_NB(1, correct_dispatch, g, Q, Wbar, wstride, cp, s)
    switch (nb) {
      case 5: return correct_dispatch<1, 5>(g, Q, Wbar, wstride, cp, s);
      case 6: return correct_dispatch<1, 6>(g, Q, Wbar, wstride, cp, s);
      case 7: return correct_dispatch<1, 7>(g, Q, Wbar, wstride, cp, s);
      case 8: return correct_dispatch<1, 8>(g, Q, Wbar, wstride, cp, s);
      case 9: return correct_dispatch<1, 9>(g, Q, Wbar, wstride, cp, s);
      case 10: return correct_dispatch<1, 10>(g, Q, Wbar, wstride, cp, s);
      case 11: return correct_dispatch<1, 11>(g, Q, Wbar, wstride, cp, s);
      case 12: return correct_dispatch<1, 12>(g, Q, Wbar, wstride, cp, s);
      default: break;
    }
  } else if (g.dim == 2) {
    RIDG_DISPATCH_NB(2, correct_dispatch, g, Q, Wbar, wstride, cp, s)
    switch (nb) {
      case 5: return correct_dispatch<2, 5>(g, Q, Wbar, wstride, cp, s);
      case 6: return correct_dispatch<2, 6>(g, Q, Wbar, wstride, cp, s);
      default: break;
    }
  } else if (g.dim == 3) {
    RIDG_DISPATCH_NB(3, correct_dispatch, g, Q, Wbar, wstride, cp, s)
    switch (nb) {
      case 5: return correct_dispatch<3, 5>(g, Q, Wbar, wstride, cp, s);
      case 6: return correct_dispatch<3, 6>(g, Q, Wbar, wstride, cp, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace ridg
