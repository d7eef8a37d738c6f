// The 3D nonlinear prediction (Sec. 2.2, eq. pred_full_system; Newton of Sec. 3) for
// Burgers' flux F_d(q) = q^2 / 2, and its correction (Sec. 2.3).
//
// One persistent CTA per SM takes regions (3 x 3 x 3 cells, 27 theta_T unknowns each) from
// an atomic counter.  Per Newton iteration, in FP64: the iterate's values at the residual's
// Gauss points (volume and the six faces of every region cell), the Rusanov face fluxes
// (speeds frozen at the initial iterate, Q^n extended in time; interior traces on the
// region boundary), the residual; then the quasi-quadrature-free Jacobian (eqs. Jacproj,
// Jacobian2: for Burgers F'(w) = w, whose projection onto Psi_p is w's own coefficients,
// contracted with the host-built triple products) written row by row into the CTA's slice of
// global memory, factorised by a right-looking LU with partial pivoting (FP64, or FP32 with
// the FP64 residual and update), and the update.  Iterations stop when
// ||dW||_inf <= tol max(1, ||W||_inf) or at the cap.  This is the paper's dense per-region
// solve (n = 27 theta_T: 432 unknowns at degree 1), not the 2D path's block elimination.
#include <cuda_runtime.h>

#include <cmath>

#include "nl3.h"
#include "ridg_internal.h"

namespace ridg {
namespace {

constexpr int kT3 = 256;
constexpr int kFlagSingular3 = 1, kFlagNonFinite3 = 2;

template <int NB>
struct D3 {
  static constexpr int THS = NB * NB * NB, THT = NB * THS, NF = NB * NB * NB, NR = 27;
  static constexpr int N = NR * THT;
  static constexpr int NQ = (3 * (NB - 1) + 2) / 2;
  static constexpr int QV = NQ * NQ * NQ * NQ, QF = NQ * NQ * NQ;
};

__device__ __forceinline__ double block_max3(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int i = 1; i < kT3 / 32; ++i) r = fmax(r, red[i]);
  __syncthreads();
  return r;
}

// region cell r (0..26, x fastest) -> offsets in {-1, 0, 1}; its neighbour across face
// (d, side) inside the region, or -1
__device__ __forceinline__ int region_nbr3(int r, int d, int side) {
  int o[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
  o[d] += side;
  if (o[d] < -1 || o[d] > 1) return -1;
  return (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
}

// k -> (bx, by, bz, a)
template <int NB>
__device__ __forceinline__ void mode_digits(int k, int* dg) {
  dg[0] = k % NB;
  dg[1] = (k / NB) % NB;
  dg[2] = (k / (NB * NB)) % NB;
  dg[3] = k / (NB * NB * NB);
}

// w at the volume point (qt, qx, qy, qz) and at the face point of face (d, side): the
// products of the 1D basis values (FP64)
template <int NB>
__device__ double eval_volume(const Nl3Dev& tb, const double* Wc, int qv) {
  using D = D3<NB>;
  const int q[4] = {qv % D::NQ, (qv / D::NQ) % D::NQ, (qv / (D::NQ * D::NQ)) % D::NQ,
                    qv / (D::NQ * D::NQ * D::NQ)};  // t, x, y, z
  double s = 0.0;
  for (int k = 0; k < D::THT; ++k) {
    int dg[4];
    mode_digits<NB>(k, dg);
    s += Wc[k] * tb.V1[dg[3] * D::NQ + q[0]] * tb.V1[dg[0] * D::NQ + q[1]] *
         tb.V1[dg[1] * D::NQ + q[2]] * tb.V1[dg[2] * D::NQ + q[3]];
  }
  return s;
}

// face point qf = qt + NQ (q1 + NQ q2) of face (d, side); e1 < e2 the transverse dimensions
template <int NB>
__device__ double eval_face(const Nl3Dev& tb, const double* Wc, int d, int side, int qf) {
  using D = D3<NB>;
  const int qt = qf % D::NQ, q1 = (qf / D::NQ) % D::NQ, q2 = qf / (D::NQ * D::NQ);
  const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  const double* tr = side > 0 ? tb.ep : tb.em;
  double s = 0.0;
  for (int k = 0; k < D::THT; ++k) {
    int dg[4];
    mode_digits<NB>(k, dg);
    s += Wc[k] * tb.V1[dg[3] * D::NQ + qt] * tb.V1[dg[e1] * D::NQ + q1] *
         tb.V1[dg[e2] * D::NQ + q2] * tr[dg[d]];
  }
  return s;
}

// trace coefficients of the cell's w on face (d, side): c[pf] over pf = (a, c1, c2)
template <int NB>
__device__ __forceinline__ double trace_coef(const Nl3Dev& tb, const double* Wc, int d, int side,
                                             int pf) {
  using D = D3<NB>;
  const int a = pf % NB, c1 = (pf / NB) % NB, c2 = pf / (NB * NB);
  const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  const double* tr = side > 0 ? tb.ep : tb.em;
  double s = 0.0;
  for (int b = 0; b < NB; ++b) {
    int dg[3];
    dg[d] = b;
    dg[e1] = c1;
    dg[e2] = c2;
    s += tr[b] * Wc[a * D::THS + dg[0] + NB * (dg[1] + NB * dg[2])];
  }
  return s;
}

template <typename T, int NB>
__global__ void __launch_bounds__(kT3, 1) newton3_kernel(const Newton3Args a) {
  using D = D3<NB>;
  constexpr int N = D::N, THT = D::THT, THS = D::THS;
  __shared__ double Ws[N], Rs[N], Qs[D::NR * THS];
  __shared__ double Fv[D::NR * D::QV];                 // F(w) at the volume points
  __shared__ double Wf[D::NR * 6 * D::QF];             // traces at the face points
  __shared__ double Fn[D::NR * 6 * D::QF];             // n . F-hat at the face points
  __shared__ double alpha[D::NR * 3];                  // frozen speed of the +d face of r
  __shared__ T rhs[N];
  __shared__ double red[kT3 / 32];
  __shared__ double redv[kT3];
  __shared__ int redi[kT3];
  __shared__ int misc[2];
  const int tid = threadIdx.x;
  T* J = (T*)((char*)a.scratch + (size_t)blockIdx.x * a.scratch_per_cta);
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const double lam8[3] = {a.lam[0] / 8.0, a.lam[1] / 8.0, a.lam[2] / 8.0};
  for (;;) {
    if (tid == 0) misc[0] = atomicAdd(a.counter, 1);
    __syncthreads();
    const long long e = misc[0];
    __syncthreads();
    if (e >= a.ncell) break;
    const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)(e / ((long long)nx * ny));
    for (int i = tid; i < D::NR * THS; i += kT3) {
      const int r = i / THS, s = i % THS;
      const int cx = (ix + r % 3 - 1 + nx) % nx, cy = (iy + (r / 3) % 3 - 1 + ny) % ny,
                cz = (iz + r / 9 - 1 + nz) % nz;
      Qs[i] = a.Q[(((long long)cz * ny + cy) * nx + cx) * THS + s];
    }
    __syncthreads();
    for (int i = tid; i < N; i += kT3) {
      const int r = i / THT, k = i % THT;
      Ws[i] = k < THS ? Qs[r * THS + k] : 0.0;  // Q^n extended constant in time
    }
    __syncthreads();
    // traces of the initial iterate -> the frozen face speeds
    for (int i = tid; i < D::NR * 6 * D::QF; i += kT3) {
      const int qf = i % D::QF, f = (i / D::QF) % 6, r = i / (6 * D::QF);
      Wf[i] = eval_face<NB>(a.tb, Ws + r * THT, f / 2, (f & 1) ? -1 : 1, qf);
    }
    __syncthreads();
    for (int i = tid; i < D::NR * 3; i += kT3) {
      const int r = i / 3, d = i % 3, r2 = region_nbr3(r, d, +1);
      double al = 0.0;
      if (r2 >= 0)
        for (int q = 0; q < D::QF; ++q)
          al = fmax(al, fmax(fabs(Wf[(r * 6 + 2 * d) * D::QF + q]),
                             fabs(Wf[(r2 * 6 + 2 * d + 1) * D::QF + q])));
      alpha[i] = al;
    }
    __syncthreads();
    int it = 0;
    bool conv = false, bad = false;
    while (!conv && !bad && it < a.max_iters) {
      // values at the residual's points
      for (int i = tid; i < D::NR * D::QV; i += kT3) {
        const double w = eval_volume<NB>(a.tb, Ws + (i / D::QV) * THT, i % D::QV);
        Fv[i] = 0.5 * w * w;
      }
      for (int i = tid; i < D::NR * 6 * D::QF; i += kT3) {
        const int qf = i % D::QF, f = (i / D::QF) % 6, r = i / (6 * D::QF);
        Wf[i] = eval_face<NB>(a.tb, Ws + r * THT, f / 2, (f & 1) ? -1 : 1, qf);
      }
      __syncthreads();
      // n . F-hat: Rusanov with the frozen speed inside the region, the interior trace's
      // flux on the region boundary
      for (int i = tid; i < D::NR * 6 * D::QF; i += kT3) {
        const int qf = i % D::QF, f = (i / D::QF) % 6, r = i / (6 * D::QF);
        const int d = f / 2, side = (f & 1) ? -1 : 1, r2 = region_nbr3(r, d, side);
        const double wo = Wf[i];
        double fn;
        if (r2 < 0) {
          fn = side * 0.5 * wo * wo;
        } else {
          const double wn = Wf[(r2 * 6 + 2 * d + (side > 0 ? 1 : 0)) * D::QF + qf];
          const double al = side > 0 ? alpha[r * 3 + d] : alpha[r2 * 3 + d];
          const double wl = side > 0 ? wo : wn, wr = side > 0 ? wn : wo;
          fn = side * (0.5 * (0.5 * wl * wl + 0.5 * wr * wr) - 0.5 * al * (wr - wl));
        }
        Fn[i] = fn;
      }
      __syncthreads();
      // the residual of eq. pred_full_system (divided by |T|, reference coordinates)
      for (int i = tid; i < N; i += kT3) {
        const int r = i / THT, k = i % THT;
        int dk[4];
        mode_digits<NB>(k, dk);
        const int s = k % THS;
        double v = 0.0;
        for (int g = 0; g < NB; ++g) v += a.tb.Mt[dk[3] * NB + g] * Ws[r * THT + g * THS + s];
        v -= a.tb.em[dk[3]] * Qs[r * THS + s];
        for (int qv = 0; qv < D::QV; ++qv) {
          const int q[4] = {qv % D::NQ, (qv / D::NQ) % D::NQ, (qv / (D::NQ * D::NQ)) % D::NQ,
                            qv / (D::NQ * D::NQ * D::NQ)};
          const double wq = a.tb.w1[q[0]] * a.tb.w1[q[1]] * a.tb.w1[q[2]] * a.tb.w1[q[3]];
          const double pt = a.tb.V1[dk[3] * D::NQ + q[0]];
          double gsum = 0.0;
          for (int d = 0; d < 3; ++d) {
            double f = pt;
            for (int e2 = 0; e2 < 3; ++e2)
              f *= (e2 == d ? a.tb.dV1 : a.tb.V1)[dk[e2] * D::NQ + q[1 + e2]];
            gsum += lam8[d] * f;
          }
          v -= wq * gsum * Fv[r * D::QV + qv];
        }
        for (int f = 0; f < 6; ++f) {
          const int d = f / 2, side = (f & 1) ? -1 : 1;
          const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
          const double trk = (side > 0 ? a.tb.ep : a.tb.em)[dk[d]];
          double fs = 0.0;
          for (int qf = 0; qf < D::QF; ++qf) {
            const int qt = qf % D::NQ, q1 = (qf / D::NQ) % D::NQ, q2 = qf / (D::NQ * D::NQ);
            fs += a.tb.w1[qt] * a.tb.w1[q1] * a.tb.w1[q2] * a.tb.V1[dk[3] * D::NQ + qt] *
                  a.tb.V1[dk[e1] * D::NQ + q1] * a.tb.V1[dk[e2] * D::NQ + q2] *
                  Fn[(r * 6 + f) * D::QF + qf];
          }
          v += lam8[d] * trk * fs;
        }
        Rs[i] = v;
        rhs[i] = (T)v;
      }
      __syncthreads();
      // the quasi-quadrature-free Jacobian, one row (r, k) per thread at a time
      for (int row = tid; row < N; row += kT3) {
        const int r = row / THT, k = row % THT;
        T* Jr = J + (size_t)row * N;
        for (int c = 0; c < N; ++c) Jr[c] = T(0);
        int dk[4];
        mode_digits<NB>(k, dk);
        const double* Wr = Ws + r * THT;
        for (int l = 0; l < THT; ++l) {
          int dl[4];
          mode_digits<NB>(l, dl);
          double v = (dk[0] == dl[0] && dk[1] == dl[1] && dk[2] == dl[2])
                         ? a.tb.Mt[dk[3] * NB + dl[3]] : 0.0;
          for (int d = 0; d < 3; ++d) {
            const double* be = a.tb.beta + (((size_t)d * THT + k) * THT + l) * THT;
            double s = 0.0;
            for (int p = 0; p < THT; ++p) s += be[p] * Wr[p];
            v -= lam8[d] * s;
          }
          Jr[r * THT + l] = (T)v;
        }
        for (int f = 0; f < 6; ++f) {
          const int d = f / 2, side = (f & 1) ? -1 : 1, r2 = region_nbr3(r, d, side);
          const int so = side > 0 ? 0 : 1;
          double go[D::NF], gn[D::NF];
          for (int pf = 0; pf < D::NF; ++pf) {
            go[pf] = trace_coef<NB>(a.tb, Wr, d, side, pf);
            gn[pf] = r2 >= 0 ? trace_coef<NB>(a.tb, Ws + r2 * THT, d, -side, pf) : 0.0;
          }
          if (r2 < 0) {
            for (int pf = 0; pf < D::NF; ++pf) go[pf] *= side;
          } else {
            const double al = side > 0 ? alpha[r * 3 + d] : alpha[r2 * 3 + d];
            // d F-hat / d w_L = (F'(w_L) + alpha) / 2, d / d w_R = (F'(w_R) - alpha) / 2;
            // n . F-hat = -F-hat on the -d face
            for (int pf = 0; pf < D::NF; ++pf) {
              go[pf] *= 0.5 * side;
              gn[pf] *= 0.5 * side;
            }
            go[0] += side > 0 ? 0.5 * al : 0.5 * al;    // +1: (w + a)/2;  -1: -(w - a)/2
            gn[0] += side > 0 ? -0.5 * al : -0.5 * al;  // +1: (w - a)/2;  -1: -(w + a)/2
          }
          for (int l = 0; l < THT; ++l) {
            const double* gm = a.tb.gamma + ((((size_t)(d * 4 + so * 2 + so) * THT + k) * THT + l) *
                                             D::NF);
            double s = 0.0;
            for (int pf = 0; pf < D::NF; ++pf) s += gm[pf] * go[pf];
            Jr[r * THT + l] += (T)(lam8[d] * s);
            if (r2 >= 0) {
              const double* gx = a.tb.gamma + ((((size_t)(d * 4 + so * 2 + (1 - so)) * THT + k) *
                                                THT + l) * D::NF);
              double s2 = 0.0;
              for (int pf = 0; pf < D::NF; ++pf) s2 += gx[pf] * gn[pf];
              Jr[r2 * THT + l] += (T)(lam8[d] * s2);
            }
          }
        }
      }
      __syncthreads();
      // right-looking LU with partial pivoting; the right-hand side follows the row swaps
      bool singular = false;
      for (int k = 0; k < N; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < N; i += kT3) {
          const double v = fabs((double)J[(size_t)i * N + k]);
          if (v > best) {
            best = v;
            bi = i;
          }
        }
        redv[tid] = best;
        redi[tid] = bi;
        __syncthreads();
        for (int o = kT3 / 2; o > 0; o >>= 1) {
          if (tid < o && (redv[tid + o] > redv[tid] ||
                          (redv[tid + o] == redv[tid] && redi[tid + o] < redi[tid]))) {
            redv[tid] = redv[tid + o];
            redi[tid] = redi[tid + o];
          }
          __syncthreads();
        }
        const int p = redi[0];
        if (!(redv[0] > 0.0)) singular = true;
        __syncthreads();
        if (p != k) {
          for (int c = tid; c < N; c += kT3) {
            const T t1 = J[(size_t)k * N + c];
            J[(size_t)k * N + c] = J[(size_t)p * N + c];
            J[(size_t)p * N + c] = t1;
          }
          if (tid == 0) {
            const T t2 = rhs[k];
            rhs[k] = rhs[p];
            rhs[p] = t2;
          }
        }
        __syncthreads();
        const T piv = J[(size_t)k * N + k];
        const T inv = singular ? T(0) : T(1) / piv;
        for (int i = k + 1 + tid; i < N; i += kT3) J[(size_t)i * N + k] *= inv;
        __syncthreads();
        const int m = N - k - 1;
        const int ty = tid / 16, tx = tid % 16;
        for (int i = k + 1 + ty; i < N; i += 16) {
          const T lik = J[(size_t)i * N + k];
          if (lik == T(0)) continue;
          T* Ji = J + (size_t)i * N;
          const T* Jk = J + (size_t)k * N;
          for (int c = k + 1 + tx; c < N; c += 16) Ji[c] -= lik * Jk[c];
        }
        (void)m;
        __syncthreads();
      }
      // L y = P r (unit lower), then U x = y
      for (int k = 0; k < N; ++k) {
        const T yk = rhs[k];
        for (int i = k + 1 + tid; i < N; i += kT3) rhs[i] -= J[(size_t)i * N + k] * yk;
        __syncthreads();
      }
      for (int k = N - 1; k >= 0; --k) {
        __syncthreads();
        const T xk = singular ? T(0) : rhs[k] / J[(size_t)k * N + k];
        __syncthreads();
        if (tid == 0) rhs[k] = xk;
        for (int i = tid; i < k; i += kT3) rhs[i] -= J[(size_t)i * N + k] * xk;
      }
      __syncthreads();
      double dn = 0.0, wn = 0.0;
      bool fin = true;
      for (int i = tid; i < N; i += kT3) {
        const double d = (double)rhs[i];
        const double w = Ws[i] - d;
        Ws[i] = w;
        fin = fin && isfinite(d) && isfinite(w);
        dn = fmax(dn, fabs(d));
        wn = fmax(wn, fabs(w));
      }
      const double nf = block_max3(fin ? 0.0 : 1.0, red);
      dn = block_max3(dn, red);
      wn = block_max3(wn, red);
      ++it;
      bad = nf > 0.0 || singular;
      conv = !bad && dn <= a.tol * fmax(1.0, wn);
      if (singular && tid == 0) atomicOr(a.stats + 2, kFlagSingular3);
    }
    for (int i = tid; i < THT; i += kT3) a.W[e * THT + i] = Ws[13 * THT + i];
    if (tid == 0) {
      if (!conv) atomicAdd(&a.stats[0], 1);
      atomicMax(&a.stats[1], it);
      atomicAdd(&a.stats[7 + (it < 15 ? it : 15)], 1);
      atomicAdd(a.iters_total, (unsigned long long)it);
      if (bad) atomicOr(a.stats + 2, kFlagNonFinite3);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// the correction: one thread per cell; every face flux is computed by both of its cells
// from the same traces in the same order (the same bits: the mass telescopes exactly)
// ---------------------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(128) nl3_correct_kernel(const Nl3Dev tb, double* __restrict__ Q,
                                                          const double* __restrict__ W, int nx,
                                                          int ny, int nz, long long ncell,
                                                          double lx, double ly, double lz) {
  using D = D3<NB>;
  constexpr int THT = D::THT, THS = D::THS;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)(e / ((long long)nx * ny));
  const double lam8[3] = {lx / 8.0, ly / 8.0, lz / 8.0};
  const double* We = W + e * THT;
  double dq[THS];
  for (int s = 0; s < THS; ++s) dq[s] = 0.0;
  // volume: sum_d lam_d / 8 sum_q w_q d_d Phi_s(q) F(w(q))
  for (int qv = 0; qv < D::QV; ++qv) {
    const int q[4] = {qv % D::NQ, (qv / D::NQ) % D::NQ, (qv / (D::NQ * D::NQ)) % D::NQ,
                      qv / (D::NQ * D::NQ * D::NQ)};
    const double wq = tb.w1[q[0]] * tb.w1[q[1]] * tb.w1[q[2]] * tb.w1[q[3]];
    const double w = eval_volume<NB>(tb, We, qv);
    const double f = 0.5 * w * w * wq;
    for (int s = 0; s < THS; ++s) {
      const int b[3] = {s % NB, (s / NB) % NB, s / (NB * NB)};
      for (int d = 0; d < 3; ++d) {
        double g = lam8[d];
        for (int e2 = 0; e2 < 3; ++e2) g *= (e2 == d ? tb.dV1 : tb.V1)[b[e2] * D::NQ + q[1 + e2]];
        dq[s] += g * f;
      }
    }
  }
  // faces: the flux at i + 1/2 from (w_i at +1, w_{i+1} at -1), at i - 1/2 from (w_{i-1} at +1,
  // w_i at -1); Rusanov with the face's largest speed
  for (int d = 0; d < 3; ++d) {
    for (int side = -1; side <= 1; side += 2) {
      int c[3] = {ix, iy, iz};
      const int nn[3] = {nx, ny, nz};
      c[d] = (c[d] + side + nn[d]) % nn[d];
      const long long en = ((long long)c[2] * ny + c[1]) * nx + c[0];
      const double* WL = side > 0 ? We : W + en * THT;
      const double* WR = side > 0 ? W + en * THT : We;
      double wl[D::QF], wr[D::QF];
      double al = 0.0;
      for (int qf = 0; qf < D::QF; ++qf) {
        wl[qf] = eval_face<NB>(tb, WL, d, +1, qf);
        wr[qf] = eval_face<NB>(tb, WR, d, -1, qf);
        al = fmax(al, fmax(fabs(wl[qf]), fabs(wr[qf])));
      }
      const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
      for (int qf = 0; qf < D::QF; ++qf) {
        const int qt = qf % D::NQ, q1 = (qf / D::NQ) % D::NQ, q2 = qf / (D::NQ * D::NQ);
        const double fh = 0.5 * (0.5 * wl[qf] * wl[qf] + 0.5 * wr[qf] * wr[qf]) -
                          0.5 * al * (wr[qf] - wl[qf]);
        const double wq = tb.w1[qt] * tb.w1[q1] * tb.w1[q2] * fh;
        for (int s = 0; s < THS; ++s) {
          const int b[3] = {s % NB, (s / NB) % NB, s / (NB * NB)};
          const double phi = (side > 0 ? tb.ep : tb.em)[b[d]] * tb.V1[b[e1] * D::NQ + q1] *
                             tb.V1[b[e2] * D::NQ + q2];
          dq[s] -= side * lam8[d] * phi * wq;
        }
      }
    }
  }
  for (int s = 0; s < THS; ++s) Q[e * THS + s] += dq[s];
}

template <int NB>
__global__ void max_speed3_kernel(const double* __restrict__ Q, long long ncell,
                                  unsigned long long* out) {
  constexpr int THS = NB * NB * NB;
  __shared__ unsigned long long sh[8];
  unsigned long long m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell * 216;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / 216;
    const int p = (int)(i % 216);
    const double x[3] = {-1.0 + 0.4 * (p % 6), -1.0 + 0.4 * ((p / 6) % 6), -1.0 + 0.4 * (p / 36)};
    double v[3][NB];
    for (int d = 0; d < 3; ++d) {
      double p0 = 1.0, p1 = x[d];
      for (int b = 0; b < NB; ++b) {
        const double pb = b == 0 ? 1.0 : (b == 1 ? x[d] : p1);
        v[d][b] = sqrt(2.0 * b + 1.0) * pb;
        if (b >= 1) {
          const double pn = ((2.0 * b + 1.0) * x[d] * p1 - b * p0) / (b + 1.0);
          p0 = p1;
          p1 = pn;
        }
      }
    }
    double w = 0.0;
    for (int s = 0; s < THS; ++s)
      w += Q[e * THS + s] * v[0][s % NB] * v[1][(s / NB) % NB] * v[2][s / (NB * NB)];
    const unsigned long long ab = (unsigned long long)__double_as_longlong(fabs(w));
    m = ab > m ? ab : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2) m = sh[w2] > m ? sh[w2] : m;
    atomicMax(out, m);
  }
}

}  // namespace

bool newton3_supported(int nb) { return nb == 2; }

size_t newton3_scratch_per_cta(int nb, bool fp32) {
  const size_t n = (size_t)27 * nb * nb * nb * nb;
  return ((n * n * (fp32 ? 4 : 8)) + 255) & ~(size_t)255;
}

cudaError_t launch_newton3(int nb, bool fp32, const Newton3Args& a, int grid, cudaStream_t s) {
  if (nb != 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (fp32)
    newton3_kernel<float, 2><<<grid, kT3, 0, s>>>(a);
  else
    newton3_kernel<double, 2><<<grid, kT3, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nl3_correct(int nb, const Nl3Dev& tb, double* Q, const double* W, const int* n,
                               long long ncell, const double* lam, cudaStream_t s) {
  if (nb != 2) return cudaErrorInvalidValue;
  nl3_correct_kernel<2><<<(unsigned)((ncell + 127) / 128), 128, 0, s>>>(
      tb, Q, W, n[0], n[1], n[2], ncell, lam[0], lam[1], lam[2]);
  return cudaGetLastError();
}

cudaError_t launch_max_speed3(int nb, const double* Q, long long ncell, unsigned long long* out,
                              cudaStream_t s) {
  if (nb != 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long work = ncell * 216;
  const unsigned blocks = (unsigned)std::min<long long>((work + 255) / 256, 4096);
  max_speed3_kernel<2><<<blocks, 256, 0, s>>>(Q, ncell, out);
  return cudaGetLastError();
}

int nl3_tables_upload(int nb, Nl3Dev& out, void* mem, size_t* bytes, cudaStream_t s) {
  const Nl3HostTables t = build_nl3_tables(nb - 1);
  const std::vector<const std::vector<double>*> parts = {&t.w1, &t.V1, &t.dV1, &t.ep, &t.em,
                                                         &t.Mt, &t.beta, &t.gamma};
  size_t total = 0;
  for (auto* p : parts) total += (p->size() * sizeof(double) + 255) & ~(size_t)255;
  if (!mem) {
    *bytes = total;
    return RIDG_OK;
  }
  if (*bytes < total) return RIDG_EINVAL;
  const double* ptrs[8];
  size_t off = 0;
  for (size_t i = 0; i < parts.size(); ++i) {
    char* dst = (char*)mem + off;
    if (cudaMemcpyAsync(dst, parts[i]->data(), parts[i]->size() * sizeof(double),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return RIDG_ECUDA;
    ptrs[i] = (const double*)dst;
    off += (parts[i]->size() * sizeof(double) + 255) & ~(size_t)255;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return RIDG_ECUDA;
  out.w1 = ptrs[0];
  out.V1 = ptrs[1];
  out.dV1 = ptrs[2];
  out.ep = ptrs[3];
  out.em = ptrs[4];
  out.Mt = ptrs[5];
  out.beta = ptrs[6];
  out.gamma = ptrs[7];
  out.nq = t.nq;
  return RIDG_OK;
}

}  // namespace ridg
