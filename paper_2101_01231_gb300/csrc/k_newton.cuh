// Newton prediction for a nonlinear flux in 2D (Sec. 3), one persistent CTA per region.
//
// For every cell the CTA solves the region system of eq. pred_full_system on the 3 x 3
// region R_i by Newton's method: the residual by tensor Gauss quadrature (FP64), the Jacobian
// quasi-quadrature-free (eqs. Jacproj, Jacobian2: F'(w) projected onto the degree-2M space-
// time basis and contracted with sparse lists of triple-product integrals), and the linear
// solve J dW = R by block elimination of the 3 x 3 block structure (corners, then edges,
// then the centre), in T = double or, for the mixed form, T = float.  The blocks live in a
// per-CTA slice of global memory (L2-resident while the CTA works on them); everything
// else of the region stays in shared memory.  Iterates start from Q^n extended constant in
// time and stop when ||dW||_inf <= tol max(1, ||W||_inf) or after max_iters.
#pragma once

#include <cuda_runtime.h>

#include "k_nlflux.cuh"
#include "ridg_internal.h"

namespace ridg {
namespace newton {

constexpr int kThreads = 256;
constexpr int kFlagSingular = 1, kFlagNonFinite = 2;

template <int NB, int MV>
struct Dims {
  static constexpr int THS = NB * NB, THT = NB * THS, BS = MV * THT;
  static constexpr int BP = (BS + 15) / 16 * 16, RR = BP / 16;
  static constexpr int NQ = (3 * (NB - 1) + 2) / 2, QV = NQ * NQ * NQ, QF = NQ * NQ;
  static constexpr int NP = 2 * NB - 1, QP = NP * NP * NP, QPF = NP * NP;
  static constexpr int MM = MV * MV;
};

constexpr size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// shared-memory layout (bytes) of one CTA
template <typename T, int NB, int MV>
struct Layout {
  using D = Dims<NB, MV>;
  static constexpr size_t oW = 0;
  static constexpr size_t oQ = up16(oW + sizeof(double) * 9 * D::BS);
  static constexpr size_t oR = up16(oQ + sizeof(double) * 9 * MV * D::THS);
  static constexpr size_t oAl = up16(oR + sizeof(double) * 9 * D::BS);
  static constexpr size_t oRed = up16(oAl + sizeof(double) * 16);
  static constexpr size_t oX = up16(oRed + sizeof(double) * 32);
  static constexpr size_t oCol = up16(oX + sizeof(T) * 9 * D::BP);
  static constexpr size_t oPerm = up16(oCol + sizeof(T) * D::BP);
  static constexpr size_t oMisc = up16(oPerm + sizeof(int) * D::BP);
  static constexpr size_t oArena = up16(oMisc + sizeof(int) * 16);
  // phase arenas
  static constexpr size_t aRes = sizeof(double) * (9 * 2 * MV * D::QV + 9 * 4 * MV * D::QF);
  static constexpr size_t aAlpha = sizeof(double) * 12 * D::QF;
  static constexpr size_t aJac =
      sizeof(double) * (MV * D::QP + 4 * D::MM * D::QP + 16 * D::MM * D::QPF);
  static constexpr size_t oSA = up16(sizeof(T) * D::BP * D::BP);
  static constexpr size_t oSB = up16(oSA + sizeof(T) * D::BP * 17);
  static constexpr size_t aLU = up16(oSB + sizeof(T) * 16 * D::BP);
  static constexpr size_t bytes = oArena + cmax(cmax(aRes, aAlpha), cmax(aJac, aLU));
};

// ---------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < kThreads / 32; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// sum_k tab[k * stride + q] w[k]
template <int N>
__device__ __forceinline__ double dotcol(const double* tab, int stride, int q, const double* w) {
  double acc = 0.0;
#pragma unroll 4
  for (int k = 0; k < N; ++k) acc = fma(tab[k * stride + q], w[k], acc);
  return acc;
}

// face index of the region's interior faces: x faces 0..5 (ry * 2 + left rx), y faces 6..11
// (6 + lower ry * 3 + rx)
__device__ __forceinline__ int region_face(int rx, int ry, int dd, int side) {
  if (dd == 0) return ry * 2 + (side > 0 ? rx : rx - 1);
  return 6 + (side > 0 ? ry : ry - 1) * 3 + rx;
}

// region neighbour across face (dd, side) of region cell r, or -1 on the region boundary
__device__ __forceinline__ int region_nbr(int r, int dd, int side) {
  const int rx = r % 3 + (dd == 0 ? side : 0), ry = r / 3 + (dd == 1 ? side : 0);
  return (rx < 0 || rx > 2 || ry < 0 || ry > 2) ? -1 : ry * 3 + rx;
}

// one pass of the tensor-product projection along `axis` (stride NP^axis) of n components,
// each a tensor of NP^ND values
template <int NP, int ND>
__device__ void proj_pass(const double* in, double* out, const double* P1, int ncomp, int axis) {
  constexpr int QN = ND == 3 ? NP * NP * NP : NP * NP;
  const int stride = axis == 0 ? 1 : (axis == 1 ? NP : NP * NP);
  for (int i = threadIdx.x; i < ncomp * QN; i += kThreads) {
    const int c = i / QN, pi = i % QN;
    const int pa = (pi / stride) % NP;
    const double* src = in + c * QN + (pi - pa * stride);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) acc = fma(P1[pa * NP + q], src[q * stride], acc);
    out[i] = acc;
  }
}

// ---------------------------------------------------------------------------------------
// Rusanov speeds, frozen at the initial iterate: alpha_f = max over the face's quadrature
// points of max(|lambda(w_L)|, |lambda(w_R)|)
// ---------------------------------------------------------------------------------------
template <int NB, int MV, int FLUX>
__device__ void frozen_alpha(const NlDev& tb, const double* Ws, double* alpha, double* tmp,
                             double g) {
  using D = Dims<NB, MV>;
  for (int i = threadIdx.x; i < 12 * D::QF; i += kThreads) {
    const int f = i / D::QF, q = i % D::QF;
    int dd, rL, rR;
    if (f < 6) {
      dd = 0;
      rL = (f / 2) * 3 + f % 2;
      rR = rL + 1;
    } else {
      dd = 1;
      rL = ((f - 6) / 3) * 3 + (f - 6) % 3;
      rR = rL + 3;
    }
    const double* tp = tb.PsiF + (size_t)(dd * 2 + 0) * D::THT * D::QF;
    const double* tm = tb.PsiF + (size_t)(dd * 2 + 1) * D::THT * D::QF;
    double wl[MV], wr[MV];
    for (int j = 0; j < MV; ++j) {
      wl[j] = dotcol<D::THT>(tp, D::QF, q, Ws + (rL * MV + j) * D::THT);
      wr[j] = dotcol<D::THT>(tm, D::QF, q, Ws + (rR * MV + j) * D::THT);
    }
    tmp[i] = fmax(nlflux::speed<FLUX>(wl, dd, g), nlflux::speed<FLUX>(wr, dd, g));
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    double m = 0.0;
    for (int q = 0; q < D::QF; ++q) m = fmax(m, tmp[threadIdx.x * D::QF + q]);
    alpha[threadIdx.x] = m;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// residual of eq. pred_full_system for the 9 region cells (FP64), divided by |T|:
//   R = time term - psi(-1) Q - volume flux + surface flux
// ---------------------------------------------------------------------------------------
template <int NB, int MV, int FLUX>
__device__ void residual(const NlDev& tb, const double* Ws, const double* Qs, double* Rs,
                         const double* alpha, double* arena, const double* lam, double g) {
  using D = Dims<NB, MV>;
  double* G = arena;                              // [9][2][MV][QV]
  double* H = arena + 9 * 2 * MV * D::QV;         // [9][4][MV][QF]
  for (int i = threadIdx.x; i < 9 * D::QV; i += kThreads) {
    const int r = i / D::QV, q = i % D::QV;
    double w[MV], f[MV];
    for (int j = 0; j < MV; ++j) w[j] = dotcol<D::THT>(tb.PsiV, D::QV, q, Ws + (r * MV + j) * D::THT);
    for (int dd = 0; dd < 2; ++dd) {
      nlflux::F<FLUX>(w, dd, f, g);
      const double s = 0.25 * lam[dd] * tb.wV[q];
      for (int j = 0; j < MV; ++j) G[((r * 2 + dd) * MV + j) * D::QV + q] = s * f[j];
    }
  }
  for (int i = threadIdx.x; i < 9 * 4 * D::QF; i += kThreads) {
    const int r = i / (4 * D::QF), f = (i / D::QF) % 4, q = i % D::QF;
    const int dd = f >> 1, si = f & 1, side = si ? -1 : 1;
    const double* to = tb.PsiF + (size_t)(dd * 2 + si) * D::THT * D::QF;
    double wo[MV], fo[MV], out[MV];
    for (int j = 0; j < MV; ++j) wo[j] = dotcol<D::THT>(to, D::QF, q, Ws + (r * MV + j) * D::THT);
    nlflux::F<FLUX>(wo, dd, fo, g);
    const int r2 = region_nbr(r, dd, side);
    if (r2 < 0) {
      for (int j = 0; j < MV; ++j) out[j] = side * fo[j];  // region boundary: interior trace
    } else {
      const double* tn = tb.PsiF + (size_t)(dd * 2 + (si ^ 1)) * D::THT * D::QF;
      double wn[MV], fn[MV];
      for (int j = 0; j < MV; ++j) wn[j] = dotcol<D::THT>(tn, D::QF, q, Ws + (r2 * MV + j) * D::THT);
      nlflux::F<FLUX>(wn, dd, fn, g);
      const double a = alpha[region_face(r % 3, r / 3, dd, side)];
      for (int j = 0; j < MV; ++j) {
        const double fh = side > 0 ? 0.5 * (fo[j] + fn[j]) - 0.5 * a * (wn[j] - wo[j])
                                   : 0.5 * (fn[j] + fo[j]) - 0.5 * a * (wo[j] - wn[j]);
        out[j] = side * fh;
      }
    }
    const double s = 0.25 * lam[dd] * tb.wF[dd * D::QF + q];
    for (int j = 0; j < MV; ++j) H[((r * 4 + f) * MV + j) * D::QF + q] = s * out[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 9 * D::BS; i += kThreads) {
    const int r = i / D::BS, j = (i / D::THT) % MV, k = i % D::THT;
    const int a = k / D::THS, s2 = k % D::THS;
    const double* w = Ws + (r * MV + j) * D::THT;
    double acc = 0.0;
    for (int c = 0; c < NB; ++c) acc = fma(tb.Mt[a * NB + c], w[c * D::THS + s2], acc);
    acc = fma(-tb.em[a], Qs[(r * MV + j) * D::THS + s2], acc);
    for (int dd = 0; dd < 2; ++dd) {
      const double* dp = tb.dPsiV + (size_t)(dd * D::THT + k) * D::QV;
      const double* gg = G + ((r * 2 + dd) * MV + j) * D::QV;
      double v = 0.0;
      for (int q = 0; q < D::QV; ++q) v = fma(dp[q], gg[q], v);
      acc -= v;
    }
    for (int f = 0; f < 4; ++f) {
      const double* pf = tb.PsiF + (size_t)(f * D::THT + k) * D::QF;
      const double* hh = H + ((r * 4 + f) * MV + j) * D::QF;
      double v = 0.0;
      for (int q = 0; q < D::QF; ++q) v = fma(pf[q], hh[q], v);
      acc += v;
    }
    Rs[i] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// quasi-quadrature-free Jacobian (eqs. Jacproj, Jacobian2) of region cell r: its diagonal
// block and its blocks towards the region neighbours, written in T to the block slots
// ---------------------------------------------------------------------------------------
template <typename T, int NB, int MV, int FLUX>
__device__ void jacobian_cell(const NlDev& tb, const NlPlan& plan, int r, const double* Ws,
                              const double* alpha, double* arena, T* slots, const double* lam,
                              double g) {
  using D = Dims<NB, MV>;
  constexpr int MM = D::MM, QP = D::QP, QPF = D::QPF, NP = D::NP, THT = D::THT, BP = D::BP;
  double* wp = arena;                    // [MV][QP]
  double* bufA = wp + MV * QP;           // [2][MM][QP]
  double* bufB = bufA + 2 * MM * QP;     // [2][MM][QP]
  double* graw = bufB + 2 * MM * QP;     // [8][MM][QPF]: own (f) and neighbour (4 + f) sides
  double* gtmp = graw + 8 * MM * QPF;    // [8][MM][QPF]
  for (int i = threadIdx.x; i < MV * QP; i += kThreads) {
    const int j = i / QP, q = i % QP;
    wp[i] = dotcol<THT>(tb.PsiAtP, QP, q, Ws + (r * MV + j) * THT);
  }
  for (int i = threadIdx.x; i < 4 * QPF; i += kThreads) {
    const int f = i / QPF, q = i % QPF;
    const int dd = f >> 1, si = f & 1, side = si ? -1 : 1;
    const double* to = tb.PsiAtFP + (size_t)(dd * 2 + si) * THT * QPF;
    double wo[MV], Jo[MM];
    for (int j = 0; j < MV; ++j) wo[j] = dotcol<THT>(to, QPF, q, Ws + (r * MV + j) * THT);
    nlflux::dF<FLUX>(wo, dd, Jo, g);
    const int r2 = region_nbr(r, dd, side);
    if (r2 < 0) {
      for (int ij = 0; ij < MM; ++ij) graw[(f * MM + ij) * QPF + q] = side * Jo[ij];
    } else {
      const double* tn = tb.PsiAtFP + (size_t)(dd * 2 + (si ^ 1)) * THT * QPF;
      double wn[MV], Jn[MM];
      for (int j = 0; j < MV; ++j) wn[j] = dotcol<THT>(tn, QPF, q, Ws + (r2 * MV + j) * THT);
      nlflux::dF<FLUX>(wn, dd, Jn, g);
      const double a = alpha[region_face(r % 3, r / 3, dd, side)];
      // d F-hat / d w_L = (F'(w_L) + alpha I) / 2, d F-hat / d w_R = (F'(w_R) - alpha I) / 2,
      // times the outward sign of the face
      for (int i2 = 0; i2 < MV; ++i2)
        for (int j2 = 0; j2 < MV; ++j2) {
          const int ij = i2 * MV + j2;
          const double dg = i2 == j2 ? a : 0.0;
          const double go = side > 0 ? 0.5 * (Jo[ij] + dg) : -0.5 * (Jo[ij] - dg);
          const double gn = side > 0 ? 0.5 * (Jn[ij] - dg) : -0.5 * (Jn[ij] + dg);
          graw[(f * MM + ij) * QPF + q] = go;
          graw[((4 + f) * MM + ij) * QPF + q] = gn;
        }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < QP; q += kThreads) {
    double w[MV], J[MM];
    for (int j = 0; j < MV; ++j) w[j] = wp[j * QP + q];
    for (int dd = 0; dd < 2; ++dd) {
      nlflux::dF<FLUX>(w, dd, J, g);
      for (int ij = 0; ij < MM; ++ij) bufA[(dd * MM + ij) * QP + q] = J[ij];
    }
  }
  __syncthreads();
  proj_pass<NP, 3>(bufA, bufB, tb.P1, 2 * MM, 0);
  proj_pass<NP, 2>(graw, gtmp, tb.P1, 8 * MM, 0);
  __syncthreads();
  proj_pass<NP, 3>(bufB, bufA, tb.P1, 2 * MM, 1);
  proj_pass<NP, 2>(gtmp, graw, tb.P1, 8 * MM, 1);
  __syncthreads();
  proj_pass<NP, 3>(bufA, bufB, tb.P1, 2 * MM, 2);
  __syncthreads();
  const double* Fp = bufB;   // [2][MM][QP]
  const double* Gp = graw;   // [8][MM][QPF]
  // diagonal block: time term - volume term + own-side face terms
  {
    T* blk = slots + (size_t)plan.slot[r * 9 + r] * BP * BP;
    int nbrs[4];
    for (int f = 0; f < 4; ++f) nbrs[f] = region_nbr(r, f >> 1, (f & 1) ? -1 : 1);
    for (int i = threadIdx.x; i < THT * THT; i += kThreads) {
      const int k = i / THT, l = i % THT;
      double acc[MM];
      for (int ij = 0; ij < MM; ++ij) acc[ij] = 0.0;
      for (int dd = 0; dd < 2; ++dd) {
        const double s = -0.25 * lam[dd];
        const int e1 = tb.bptr[dd][i + 1];
        for (int e = tb.bptr[dd][i]; e < e1; ++e) {
          const double v = s * tb.bval[dd][e];
          const double* fp = Fp + dd * MM * QP + tb.bp[dd][e];
          for (int ij = 0; ij < MM; ++ij) acc[ij] = fma(v, fp[ij * QP], acc[ij]);
        }
      }
      for (int f = 0; f < 4; ++f) {
        const int dd = f >> 1, si = f & 1, gi = dd * 4 + si * 2 + si;
        const double s = 0.25 * lam[dd];
        const int e1 = tb.gptr[gi][i + 1];
        for (int e = tb.gptr[gi][i]; e < e1; ++e) {
          const double v = s * tb.gval[gi][e];
          const double* gp = Gp + f * MM * QPF + tb.gp[gi][e];
          for (int ij = 0; ij < MM; ++ij) acc[ij] = fma(v, gp[ij * QPF], acc[ij]);
        }
      }
      if (k % D::THS == l % D::THS) {
        const double mt = tb.Mt[(k / D::THS) * NB + l / D::THS];
        for (int j = 0; j < MV; ++j) acc[j * MV + j] += mt;
      }
      for (int i2 = 0; i2 < MV; ++i2)
        for (int j2 = 0; j2 < MV; ++j2)
          blk[(size_t)(i2 * THT + k) * BP + j2 * THT + l] = (T)acc[i2 * MV + j2];
    }
    // blocks towards the region neighbours: neighbour-side face terms
    for (int f = 0; f < 4; ++f) {
      const int r2 = nbrs[f];
      if (r2 < 0) continue;
      const int dd = f >> 1, si = f & 1, gi = dd * 4 + si * 2 + (si ^ 1);
      const double s = 0.25 * lam[dd];
      T* ob = slots + (size_t)plan.slot[r * 9 + r2] * BP * BP;
      for (int i = threadIdx.x; i < THT * THT; i += kThreads) {
        const int k = i / THT, l = i % THT;
        double acc[MM];
        for (int ij = 0; ij < MM; ++ij) acc[ij] = 0.0;
        const int e1 = tb.gptr[gi][i + 1];
        for (int e = tb.gptr[gi][i]; e < e1; ++e) {
          const double v = s * tb.gval[gi][e];
          const double* gp = Gp + (4 + f) * MM * QPF + tb.gp[gi][e];
          for (int ij = 0; ij < MM; ++ij) acc[ij] = fma(v, gp[ij * QPF], acc[ij]);
        }
        for (int i2 = 0; i2 < MV; ++i2)
          for (int j2 = 0; j2 < MV; ++j2)
            ob[(size_t)(i2 * THT + k) * BP + j2 * THT + l] = (T)acc[i2 * MV + j2];
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// dense block kernels of the elimination (T), all BP x BP row-major with zero padding
// ---------------------------------------------------------------------------------------
// In-place Gauss-Jordan inverse of the leading BS x BS part of S (row stride BP), partial
// pivoting by rows; the row interchanges are undone on the columns at the end.
template <typename T, int BS, int BP>
__device__ void gauss_jordan(T* S, T* colf, int* perm, int* misc, int* flags) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int c = 0; c < BS; ++c) {
    if (tid < 32) {
      T best = T(-1);
      int bi = c;
      for (int i = c + lane; i < BS; i += 32) {
        const T v = fabs(S[i * BP + c]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        misc[1] = bi;
        perm[c] = bi;
        if (!(best > T(0))) atomicOr(flags, kFlagSingular);
      }
    }
    __syncthreads();
    const int p = misc[1];
    if (p != c)
      for (int j = tid; j < BS; j += kThreads) {
        const T t = S[c * BP + j];
        S[c * BP + j] = S[p * BP + j];
        S[p * BP + j] = t;
      }
    __syncthreads();
    for (int i = tid; i < BS; i += kThreads) colf[i] = S[i * BP + c];
    __syncthreads();
    const T ipiv = T(1) / colf[c];
    for (int j = tid; j < BS; j += kThreads) S[c * BP + j] = j == c ? ipiv : S[c * BP + j] * ipiv;
    __syncthreads();
    for (int idx = tid; idx < BS * BS; idx += kThreads) {
      const int i = idx / BS, j = idx % BS;
      if (i != c) {
        const T v = j == c ? T(0) : S[i * BP + j];
        S[i * BP + j] = v - colf[i] * S[c * BP + j];
      }
    }
    __syncthreads();
  }
  for (int c = BS - 1; c >= 0; --c) {
    const int p = perm[c];
    if (p != c)
      for (int i = tid; i < BS; i += kThreads) {
        const T t = S[i * BP + c];
        S[i * BP + c] = S[i * BP + p];
        S[i * BP + p] = t;
      }
    __syncthreads();
  }
}

// C = (overwrite ? 0 : C) - A B  (A, B, C in global memory)
template <typename T, int BP, int RR>
__device__ void gemm_sub(T* C, const T* A, const T* B, bool overwrite, T* sA, T* sB) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RR][RR];
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < BP; k0 += 16) {
    for (int i = threadIdx.x; i < BP * 16; i += kThreads) {
      const int row = i >> 4, kk = i & 15;
      sA[row * 17 + kk] = A[(size_t)row * BP + k0 + kk];
      const int kr = i / BP, col = i % BP;
      sB[kr * BP + col] = B[(size_t)(k0 + kr) * BP + col];
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      T av[RR], bv[RR];
#pragma unroll
      for (int a = 0; a < RR; ++a) av[a] = sA[(ty + 16 * a) * 17 + kk];
#pragma unroll
      for (int b = 0; b < RR; ++b) bv[b] = sB[kk * BP + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < RR; ++a)
#pragma unroll
        for (int b = 0; b < RR; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) {
      T* c = C + (size_t)(ty + 16 * a) * BP + tx + 16 * b;
      *c = (overwrite ? T(0) : *c) - acc[a][b];
    }
  __syncthreads();
}

// B = S B in place (S in shared memory, B in global memory)
template <typename T, int BP, int RR>
__device__ void gemm_left_inplace(const T* S, T* B, T* sB) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RR][RR];
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < BP; k0 += 16) {
    for (int i = threadIdx.x; i < BP * 16; i += kThreads) {
      const int kr = i / BP, col = i % BP;
      sB[kr * BP + col] = B[(size_t)(k0 + kr) * BP + col];
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      T av[RR], bv[RR];
#pragma unroll
      for (int a = 0; a < RR; ++a) av[a] = S[(ty + 16 * a) * BP + k0 + kk];
#pragma unroll
      for (int b = 0; b < RR; ++b) bv[b] = sB[kk * BP + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < RR; ++a)
#pragma unroll
        for (int b = 0; b < RR; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) B[(size_t)(ty + 16 * a) * BP + tx + 16 * b] = acc[a][b];
  __syncthreads();
}

// y -= M x for the first BS rows (M global, x and y shared); one warp per row
template <typename T, int BS, int BP>
__device__ void matvec_sub(const T* M, const T* x, T* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < BS; r += kThreads / 32) {
    T s = T(0);
    for (int c = lane; c < BS; c += 32) s = fma(M[(size_t)r * BP + c], x[c], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[r] -= s;
  }
  __syncthreads();
}

// Solve J x = b by block elimination in the plan's order; b in xs (9 x BP), x returned there.
template <typename T, int BS, int BP, int RR>
__device__ void block_solve(T* slots, const NlPlan& plan, T* xs, T* S, T* sA, T* sB, T* colf,
                            int* perm, int* misc, int* flags) {
  const int tid = threadIdx.x;
  for (int t = 0; t < 9; ++t) {
    const int k = plan.order[t];
    const T* Akk = slots + (size_t)plan.slot[k * 9 + k] * BP * BP;
    for (int i = tid; i < BP * BP; i += kThreads) S[i] = Akk[i];
    __syncthreads();
    gauss_jordan<T, BS, BP>(S, colf, perm, misc, flags);
    T* xk = xs + k * BP;
    if (tid < BS) {
      T acc = T(0);
      for (int c = 0; c < BS; ++c) acc = fma(S[tid * BP + c], xk[c], acc);
      colf[tid] = acc;
    }
    __syncthreads();
    if (tid < BS) xk[tid] = colf[tid];
    __syncthreads();
    const int nn = plan.nn[t];
    for (int a = 0; a < nn; ++a) {
      const int j = plan.nbr[t][a];
      gemm_left_inplace<T, BP, RR>(S, slots + (size_t)plan.slot[k * 9 + j] * BP * BP, sB);
    }
    for (int a = 0; a < nn; ++a) {
      const int i = plan.nbr[t][a];
      const T* Aik = slots + (size_t)plan.slot[i * 9 + k] * BP * BP;
      matvec_sub<T, BS, BP>(Aik, xk, xs + i * BP);
      for (int b = 0; b < nn; ++b) {
        const int j = plan.nbr[t][b];
        gemm_sub<T, BP, RR>(slots + (size_t)plan.slot[i * 9 + j] * BP * BP, Aik,
                            slots + (size_t)plan.slot[k * 9 + j] * BP * BP, plan.first[t][a][b] != 0,
                            sA, sB);
      }
    }
  }
  for (int t = 8; t >= 0; --t) {
    const int k = plan.order[t];
    for (int a = 0; a < plan.nn[t]; ++a) {
      const int j = plan.nbr[t][a];
      matvec_sub<T, BS, BP>(slots + (size_t)plan.slot[k * 9 + j] * BP * BP, xs + j * BP, xs + k * BP);
    }
  }
}

// ---------------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------------
template <typename T, int NB, int MV, int FLUX>
__global__ void __launch_bounds__(kThreads, 1) newton_kernel(const NewtonArgs a) {
  using D = Dims<NB, MV>;
  using L = Layout<T, NB, MV>;
  extern __shared__ __align__(16) unsigned char smem[];
  double* Ws = (double*)(smem + L::oW);
  double* Qs = (double*)(smem + L::oQ);
  double* Rs = (double*)(smem + L::oR);
  double* alpha = (double*)(smem + L::oAl);
  double* red = (double*)(smem + L::oRed);
  T* xs = (T*)(smem + L::oX);
  T* colf = (T*)(smem + L::oCol);
  int* perm = (int*)(smem + L::oPerm);
  int* misc = (int*)(smem + L::oMisc);
  unsigned char* arena = smem + L::oArena;
  T* S = (T*)arena;
  T* sA = (T*)(arena + L::oSA);
  T* sB = (T*)(arena + L::oSB);
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  T* slots = (T*)((char*)a.scratch + (size_t)blockIdx.x * a.scratch_per_cta);
  int* flags = a.stats + 2;

  for (;;) {
    if (tid == 0) misc[0] = atomicAdd(a.counter, 1);
    __syncthreads();
    const long long e = misc[0];
    __syncthreads();
    if (e >= a.ncell) break;
    const int ix = (int)(e % nx), iy = (int)(e / nx);
    for (int i = tid; i < 9 * MV * D::THS; i += kThreads) {
      const int r = i / (MV * D::THS), rem = i % (MV * D::THS);
      const long long c = (long long)((iy + r / 3 - 1 + ny) % ny) * nx + (ix + r % 3 - 1 + nx) % nx;
      Qs[i] = a.Q[c * MV * D::THS + rem];
    }
    __syncthreads();
    for (int i = tid; i < 9 * D::BS; i += kThreads) {
      const int r = i / D::BS, j = (i / D::THT) % MV, k = i % D::THT;
      Ws[i] = k < D::THS ? Qs[(r * MV + j) * D::THS + k] : 0.0;  // Q^n extended in time
    }
    __syncthreads();
    frozen_alpha<NB, MV, FLUX>(a.tb, Ws, alpha, (double*)arena, a.gamma);
    int it = 0;
    bool conv = false, bad = false;
    while (it < a.max_iters && !conv && !bad) {
      residual<NB, MV, FLUX>(a.tb, Ws, Qs, Rs, alpha, (double*)arena, a.lam, a.gamma);
      for (int r = 0; r < 9; ++r)
        jacobian_cell<T, NB, MV, FLUX>(a.tb, a.plan, r, Ws, alpha, (double*)arena, slots, a.lam,
                                       a.gamma);
      for (int i = tid; i < 9 * D::BP; i += kThreads) {
        const int r = i / D::BP, c = i % D::BP;
        xs[i] = c < D::BS ? (T)Rs[r * D::BS + c] : T(0);
      }
      __syncthreads();
      block_solve<T, D::BS, D::BP, D::RR>(slots, a.plan, xs, S, sA, sB, colf, perm, misc, flags);
      double dn = 0.0, wn = 0.0;
      bool fin = true;
      for (int i = tid; i < 9 * D::BS; i += kThreads) {
        const double d = (double)xs[(i / D::BS) * D::BP + i % D::BS];
        const double w = Ws[i] - d;
        Ws[i] = w;
        fin = fin && isfinite(d) && isfinite(w);
        dn = fmax(dn, fabs(d));
        wn = fmax(wn, fabs(w));
      }
      const double nf = block_max(fin ? 0.0 : 1.0, red);
      dn = block_max(dn, red);
      wn = block_max(wn, red);
      ++it;
      bad = nf > 0.0;
      conv = !bad && dn <= a.tol * fmax(1.0, wn);
    }
    for (int i = tid; i < D::BS; i += kThreads) a.W[e * D::BS + i] = Ws[4 * D::BS + i];
    if (tid == 0) {
      if (!conv) atomicAdd(&a.stats[0], 1);
      atomicMax(&a.stats[1], it);
      if (bad) atomicOr(flags, kFlagNonFinite);
    }
    __syncthreads();
  }
}

template <typename T, int NB, int MV, int FLUX>
cudaError_t launch_one(const NewtonArgs& a, int grid, cudaStream_t s) {
  using L = Layout<T, NB, MV>;
  static_assert(L::bytes <= 232448, "Newton kernel shared memory above the per-CTA limit");
  cudaError_t e = cudaFuncSetAttribute(newton_kernel<T, NB, MV, FLUX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  newton_kernel<T, NB, MV, FLUX><<<grid, kThreads, L::bytes, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_typed(int nb, int m, int kind, const NewtonArgs& a, int grid, cudaStream_t s) {
  if (kind == RIDG_FLUX_BURGERS && m == 1) {
    switch (nb) {
      case 2: return launch_one<T, 2, 1, RIDG_FLUX_BURGERS>(a, grid, s);
      case 3: return launch_one<T, 3, 1, RIDG_FLUX_BURGERS>(a, grid, s);
      case 4: return launch_one<T, 4, 1, RIDG_FLUX_BURGERS>(a, grid, s);
      case 5: return launch_one<T, 5, 1, RIDG_FLUX_BURGERS>(a, grid, s);
      default: break;
    }
  } else if (kind == RIDG_FLUX_EULER && m == 4) {
    switch (nb) {
      case 2: return launch_one<T, 2, 4, RIDG_FLUX_EULER>(a, grid, s);
      case 3: return launch_one<T, 3, 4, RIDG_FLUX_EULER>(a, grid, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace newton
}  // namespace ridg
