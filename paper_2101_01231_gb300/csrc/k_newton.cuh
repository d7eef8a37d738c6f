// Newton prediction for a nonlinear flux in 2D (Sec. 3), one persistent CTA per region.
//
// For every cell the CTA solves the region system of eq. pred_full_system on the 3 x 3
// region R_i by Newton's method:
//  * the residual by tensor Gauss quadrature, always in FP64 (it defines the fixed point);
//  * the Jacobian quasi-quadrature-free (eqs. Jacproj, Jacobian2): F'(w) projected onto the
//    degree-2M space-time basis by a tensor-product projection, then contracted with the
//    triple-product lists merged per (k, l) pair; in T;
//  * the linear solve J dW = R by block elimination of the 3 x 3 block structure (corners,
//    edges, centre): every pivot block inverted by Gauss-Jordan with implicit row pivoting
//    on a register-resident tile, the other blocks updated by register-tiled GEMMs; in T.
// T = double (RIDG_PREC_FP64) or float (RIDG_PREC_MIXED_FP32: FP32 Jacobian and solves,
// FP64 residual and iterate).  With TC (RIDG_PREC_MIXED_TF32, T = float) the block updates
// of the elimination -- U_kj = A_kk^-1 A_kj and the Schur complements A_ij -= A_ik U_kj --
// run on the 5th-generation tensor cores (tcgen05.mma kind::tf32, FP32 accumulation in
// TMEM): every block is kept in the MMA's canonical K-major layout, the blocks right of the
// pivot transposed, so that each product reads its two operands with plain bulk copies and
// writes its result in the layout the next product reads.  The blocks live in a per-CTA
// slice of global memory; the rest of the region stays in shared memory.  Iterates start from Q^n extended constant in
// time and stop when ||dW||_inf <= tol max(1, ||W||_inf) or after max_iters.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "k_nlflux.cuh"
#include "k_tcgen05.cuh"
#include "ridg_internal.h"

namespace ridg {
namespace newton {

constexpr int kThreads = 256;
constexpr int kFlagSingular = 1, kFlagNonFinite = 2, kFlagTimeout = 4;

template <int NB, int MV>
struct Dims {
  static constexpr int THS = NB * NB, THT = NB * THS, BS = MV * THT;
  static constexpr int BP = (BS + 15) / 16 * 16, RR = BP / 16;
  static constexpr int NQ = (3 * (NB - 1) + 2) / 2, QV = NQ * NQ * NQ, QF = NQ * NQ;
  static constexpr int NP = 2 * NB - 1, QP = NP * NP * NP, QPF = NP * NP;
  static constexpr int MM = MV * MV;
  static constexpr int CG = MV == 1 ? 9 : 1;              // cells assembled per list pass
  static constexpr int FAS = (2 * QP + 8 * QPF) * MM;     // projected arrays of one cell
  static constexpr int PB = 2 * MM * QP > 8 * MM * QPF ? 2 * MM * QP : 8 * MM * QPF;
};

// scratch sizes (doubles) of the residual's buffers
template <int NB, int MV>
struct ResBufs {
  using D = Dims<NB, MV>;
  static constexpr int C = 9 * MV, NQ = D::NQ, QV = D::QV, QF = D::QF;
  static constexpr int c2max(int a, int b) { return a > b ? a : b; }
  static constexpr int R1 = c2max(C * QV, 4 * C * QF);  // G_d; the faces' traces and fluxes
  static constexpr int R2 = c2max(c2max(C * NB * NB * NQ, C * QV), c2max(2 * C * NB * NB, 2 * C * NQ * NB));
  static constexpr int R3 = c2max(c2max(C * NB * NQ * NQ, C * NQ * NQ * NB), 2 * C * NB * NQ);
  static constexpr int R4 = C * D::THT;                 // volume term
  static constexpr int R5 = 4 * C * NB * NB;            // face terms, per face
  static constexpr int total = R1 + R2 + R3 + R4 + R5;
};

constexpr size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// packed assembly-list entries (see NlDev)
template <typename T>
struct Ent;
template <>
struct Ent<double> {
  int off, pad;
  double c;
};
template <>
struct Ent<float> {
  int off;
  float c;
};

// per-precision table pointers
template <typename T>
struct Tab;
template <>
struct Tab<double> {
  static __device__ __forceinline__ const double* Mt(const NlDev& t) { return t.Mt; }
  static __device__ __forceinline__ const double* PsiAtP(const NlDev& t) { return t.PsiAtP; }
  static __device__ __forceinline__ const double* PsiAtFP(const NlDev& t) { return t.PsiAtFP; }
  static __device__ __forceinline__ const double* P1(const NlDev& t) { return t.P1; }
  static __device__ __forceinline__ const Ent<double>* dent(const NlDev& t) {
    return (const Ent<double>*)t.dent_d;
  }
  static __device__ __forceinline__ const Ent<double>* oent(const NlDev& t, int f) {
    return (const Ent<double>*)t.oent_d[f];
  }
};
template <>
struct Tab<float> {
  static __device__ __forceinline__ const float* Mt(const NlDev& t) { return t.Mt_f; }
  static __device__ __forceinline__ const float* PsiAtP(const NlDev& t) { return t.PsiAtP_f; }
  static __device__ __forceinline__ const float* PsiAtFP(const NlDev& t) { return t.PsiAtFP_f; }
  static __device__ __forceinline__ const float* P1(const NlDev& t) { return t.P1_f; }
  static __device__ __forceinline__ const Ent<float>* dent(const NlDev& t) {
    return (const Ent<float>*)t.dent_f;
  }
  static __device__ __forceinline__ const Ent<float>* oent(const NlDev& t, int f) {
    return (const Ent<float>*)t.oent_f[f];
  }
};

// tensor-core block products: K-slices of 16 columns, a ring of kStages slices of both
// operands (the A operand followed by (128 - BP) spare rows, read by the M = 128 MMA into
// accumulator lanes that are never used)
constexpr int kStages = 4, kKS = 16;
template <int BP>
struct TcDims {
  static constexpr uint32_t SL = kKS * BP * 4;          // one operand's K-slice (bytes)
  static constexpr uint32_t PAD = (128 - BP) * 16;      // rows BP .. 127 of the A operand
  static constexpr uint32_t STAGE = (2 * SL + PAD + 127) & ~127u;
  static constexpr int NS = BP / kKS;                   // K-slices per product
};

// the instance of the region a CTA is solving, kept in shared memory (read where needed,
// so that it holds no registers through the Newton iteration)
struct RegionCtx {
  double lam[2];
  double* W;
  int* stats;
  unsigned long long* itot;
  long long e;  // the region (cell) within its instance
};
static_assert(sizeof(RegionCtx) <= 64, "RegionCtx slot");

// shared-memory layout (bytes) of one CTA
template <typename T, int NB, int MV, bool TC = false>
struct Layout {
  using D = Dims<NB, MV>;
  static constexpr int NBUF = sizeof(T) == 4 ? 2 : 1;     // GEMM staging buffers
  static constexpr size_t oW = 0;
  static constexpr size_t oQ = up16(oW + sizeof(double) * 9 * D::BS);
  static constexpr size_t oR = up16(oQ + sizeof(double) * 9 * MV * D::THS);
  static constexpr size_t oAl = up16(oR + sizeof(double) * 9 * D::BS);
  static constexpr size_t oRed = up16(oAl + sizeof(double) * 16);
  static constexpr size_t oX = up16(oRed + sizeof(double) * 32);
  static constexpr size_t oCol = up16(oX + sizeof(T) * 9 * D::BP);
  static constexpr size_t oRow = up16(oCol + sizeof(T) * 2 * D::BP);
  static constexpr size_t oProw = up16(oRow + sizeof(T) * 2 * D::BP);
  static constexpr size_t oRank = up16(oProw + sizeof(int) * D::BP);
  static constexpr size_t oMisc = up16(oRank + sizeof(int) * D::BP);
  // the current region's instance (RegionCtx)
  static constexpr size_t oCtx = up16(oMisc + sizeof(int) * 16);
  // mbarriers of the tensor-core products: full[kStages], empty[kStages], acc; TMEM address
  static constexpr size_t oBar = up16(oCtx + 64);
  static constexpr size_t oTmem = oBar + 8 * (2 * kStages + 1);
  static constexpr size_t oArena = TC ? ((oTmem + 4 + 127) & ~(size_t)127) : up16(oCtx + 64);
  // phase arenas
  static constexpr size_t aRes = sizeof(double) * ResBufs<NB, MV>::total;
  static constexpr size_t aAlpha = sizeof(double) * 12 * D::QF;
  // FP32 assembly of one conserved variable: one cell at a time, its triple products
  // contracted one dimension at a time (assemble_cell_sf); else CG cells per list pass
  static constexpr bool SF = sizeof(T) == 4 && MV == 1;
  static constexpr int CGL = SF ? 1 : D::CG;
  static constexpr size_t oJW = up16(sizeof(T) * CGL * D::FAS);       // after the FA arrays
  static constexpr size_t oJB0 = up16(oJW + sizeof(T) * MV * D::QP);
  static constexpr size_t oJB1 = up16(oJB0 + sizeof(T) * D::PB);
  static constexpr size_t aJac = up16(oJB1 + sizeof(T) * D::PB);
  // the sum-factorised assembly's buffers, where the projection's were (after FA)
  static constexpr int NB2 = NB * NB, NP2 = D::NP * D::NP;
  static constexpr int SFN = 2 * NP2 * NB2 + D::NP * NB2 * NB2 + 4 * D::NP * NB2 + NB2 * NB2;
  static constexpr size_t aSF = SF ? up16(oJW + sizeof(T) * SFN) : 0;
  static constexpr size_t oSA = up16(sizeof(T) * D::BP * D::BP);
  static constexpr size_t oSB = up16(oSA + sizeof(T) * NBUF * D::BP * 17);
  static constexpr size_t aLU = TC ? (size_t)kStages * TcDims<D::BP>::STAGE
                                   : up16(oSB + sizeof(T) * NBUF * 16 * D::BP);
  static constexpr size_t bytes = oArena + cmax(cmax(aRes, aAlpha), cmax(cmax(aJac, aSF), aLU));
  // CTAs per SM: two where their shared memory fits (FP32 solves), else one
  static constexpr int MINB = (sizeof(T) == 4 && 2 * (bytes + 1024) <= 233472) ? 2 : 1;
};

// offset of element (r, c) of a BP x BP block in its storage.  Plain forms: row-major.
// Tensor-core form: the canonical K-major core-matrix order of the MMA operands -- 16-byte
// rows of 4 consecutive columns, the BP rows of one 4-column chunk contiguous, the chunks in
// column order -- of the block, or of its transpose when tr is set.
template <bool TC, int BP>
__device__ __forceinline__ int bidx(int r, int c, bool tr = false) {
  if constexpr (!TC) {
    return r * BP + c;
  } else {
    const int R = tr ? c : r, C = tr ? r : c;
    return ((C >> 2) * BP + R) * 4 + (C & 3);
  }
}

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
template <int N, typename S, typename U>
__device__ __forceinline__ S dotcol(const S* tab, int stride, int q, const U* w) {
  S acc = S(0);
#pragma unroll 4
  for (int k = 0; k < N; ++k) acc = fma(tab[k * stride + q], (S)w[k], acc);
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

// one pass of the tensor-product projection along `axis` (stride NP^axis) of ncomp
// component tensors of NP^ND values: out[c][.] = sum_q P1[p][q] in[c][..q..]
template <int NP, int ND, typename T>
__device__ void proj_pass(const T* in, T* out, const T* P1, int ncomp, int axis) {
  constexpr int QN = ND == 3 ? NP * NP * NP : NP * NP;
  const int stride = axis == 0 ? 1 : (axis == 1 ? NP : NP * NP);
  for (int i = threadIdx.x; i < ncomp * QN; i += kThreads) {
    const int c = i / QN, pi = i % QN;
    const int pa = (pi / stride) % NP;
    const T* src = in + c * QN + (pi - pa * stride);
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < NP; ++q) acc = fma(P1[pa * NP + q], src[q * stride], acc);
    out[i] = acc;
  }
}

// the last pass, along the slowest axis, written point-major (m x m matrices contiguous)
// with a per-component-group scale: out[(pbase(c) + p) * MM + ij] = scale(c) sum_q ...
template <int NP, int ND, int MM, typename T>
__device__ void proj_last(const T* in, T* out, const T* P1, int nsets, int set_base_stride,
                          int set_base0, const T* scale) {
  constexpr int QN = ND == 3 ? NP * NP * NP : NP * NP;
  constexpr int stride = ND == 3 ? NP * NP : NP;
  for (int i = threadIdx.x; i < nsets * MM * QN; i += kThreads) {
    const int c = i / QN, pi = i % QN;
    const int set = c / MM, ij = c % MM;
    const int pa = pi / stride;
    const T* src = in + c * QN + (pi - pa * stride);
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < NP; ++q) acc = fma(P1[pa * NP + q], src[q * stride], acc);
    out[(set_base0 + set * set_base_stride + pi) * MM + ij] = scale[set] * acc;
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
//   R = time term - psi(-1) Q - volume flux + surface flux,
// with the tensor-product quadrature evaluated by sum factorisation: every pass contracts
// one axis of a [component][t][y][x] tensor with a 1D table.
// ---------------------------------------------------------------------------------------
// out[c][o2][o1][o0] (+)= sum_i M[o_ax * ldm + i] in[c][..i..]: axis AX (0 = fastest) of the
// input [A2][A1][A0] contracted into NO outputs; components c >= csplit use M2 instead of M1
template <int A2, int A1, int A0, int AX, int NO, bool ACC = false>
__device__ void apply1d(const double* in, double* out, const double* M1, const double* M2,
                        int ldm, int ncomp, int csplit) {
  constexpr int NI = AX == 0 ? A0 : (AX == 1 ? A1 : A2);
  constexpr int O2 = AX == 2 ? NO : A2, O1 = AX == 1 ? NO : A1, O0 = AX == 0 ? NO : A0;
  constexpr int OSZ = O2 * O1 * O0, ISZ = A2 * A1 * A0;
  constexpr int IST = AX == 0 ? 1 : (AX == 1 ? A0 : A0 * A1);
  for (int idx = threadIdx.x; idx < ncomp * OSZ; idx += kThreads) {
    const int c = idx / OSZ, o = idx % OSZ;
    const int i2 = o / (O1 * O0), i1 = (o / O0) % O1, i0 = o % O0;
    const int oa = AX == 0 ? i0 : (AX == 1 ? i1 : i2);
    const int base = c * ISZ + (AX == 2 ? 0 : i2 * A1 * A0) + (AX == 1 ? 0 : i1 * A0) + (AX == 0 ? 0 : i0);
    const double* M = (c >= csplit ? M2 : M1) + oa * ldm;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i) acc = fma(M[i], in[base + i * IST], acc);
    if (ACC)
      out[idx] += acc;
    else
      out[idx] = acc;
  }
}

template <int NB, int MV, int FLUX>
__device__ void residual(const NlDev& tb, const double* Ws, const double* Qs, double* Rs,
                         const double* alpha, double* arena, const double* lam, double g) {
  using D = Dims<NB, MV>;
  using B = ResBufs<NB, MV>;
  constexpr int C = B::C, NQ = D::NQ, QV = D::QV, QF = D::QF, THT = D::THT, THS = D::THS;
  double* r1 = arena;
  double* r2 = r1 + B::R1;
  double* r3 = r2 + B::R2;
  double* rv = r3 + B::R3;
  double* k2 = rv + B::R4;
  // ---- values of W at the volume points: x, y, t passes ----
  apply1d<NB, NB, NB, 0, NQ>(Ws, r2, tb.V1T, tb.V1T, NB, C, C);
  __syncthreads();
  apply1d<NB, NB, NQ, 1, NQ>(r2, r3, tb.V1T, tb.V1T, NB, C, C);
  __syncthreads();
  apply1d<NB, NQ, NQ, 2, NQ>(r3, r2, tb.V1T, tb.V1T, NB, C, C);  // w: [c][qt][qy][qx]
  __syncthreads();
  // ---- volume term: sum_q d_d Psi_k w_q F_d, per direction ----
  for (int dd = 0; dd < 2; ++dd) {
    for (int i = threadIdx.x; i < 9 * QV; i += kThreads) {
      const int r = i / QV, q = i % QV;
      double w[MV], f[MV];
      for (int j = 0; j < MV; ++j) w[j] = r2[(r * MV + j) * QV + q];
      nlflux::F<FLUX>(w, dd, f, g);
      const double s = 0.25 * lam[dd] * tb.wV[q];
      for (int j = 0; j < MV; ++j) r1[(r * MV + j) * QV + q] = s * f[j];
    }
    __syncthreads();
    const double* Mx = dd == 0 ? tb.dV1 : tb.V1;
    const double* My = dd == 0 ? tb.V1 : tb.dV1;
    apply1d<NQ, NQ, NQ, 0, NB>(r1, r3, Mx, Mx, NQ, C, C);
    __syncthreads();
    apply1d<NQ, NQ, NB, 1, NB>(r3, r1, My, My, NQ, C, C);
    __syncthreads();
    if (dd == 0)
      apply1d<NQ, NB, NB, 2, NB, false>(r1, rv, tb.V1, tb.V1, NQ, C, C);
    else
      apply1d<NQ, NB, NB, 2, NB, true>(r1, rv, tb.V1, tb.V1, NQ, C, C);
    __syncthreads();
  }
  // ---- faces, per direction: traces of both sides, Rusanov / interior fluxes, then the
  // face basis (psi_a(t) phi_bo(other) phi_bd(+-1)) ----
  for (int dd = 0; dd < 2; ++dd) {
    double* trF = r1;              // [side][c][qt][qo]
    double* H = r1 + 2 * C * QF;   // [side][c][qt][qo]
    double* Z = r2;                // [side][c][a][bo]
    double* Zo = r3;               // [side][c][a][qo]
    if (dd == 0) {
      apply1d<NB, NB, NB, 0, 1>(Ws, Z, tb.ep1, tb.ep1, NB, C, C);
      apply1d<NB, NB, NB, 0, 1>(Ws, Z + C * NB * NB, tb.em1, tb.em1, NB, C, C);
      __syncthreads();
      apply1d<NB, NB, 1, 1, NQ>(Z, Zo, tb.V1T, tb.V1T, NB, 2 * C, 2 * C);
      __syncthreads();
      apply1d<NB, NQ, 1, 2, NQ>(Zo, trF, tb.V1T, tb.V1T, NB, 2 * C, 2 * C);
    } else {
      apply1d<NB, NB, NB, 1, 1>(Ws, Z, tb.ep1, tb.ep1, NB, C, C);
      apply1d<NB, NB, NB, 1, 1>(Ws, Z + C * NB * NB, tb.em1, tb.em1, NB, C, C);
      __syncthreads();
      apply1d<NB, 1, NB, 0, NQ>(Z, Zo, tb.V1T, tb.V1T, NB, 2 * C, 2 * C);
      __syncthreads();
      apply1d<NB, 1, NQ, 2, NQ>(Zo, trF, tb.V1T, tb.V1T, NB, 2 * C, 2 * C);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * 9 * QF; i += kThreads) {
      const int si = i / (9 * QF), r = (i / QF) % 9, q = i % QF;
      const int side = si ? -1 : 1;
      double wo[MV], fo[MV], out[MV];
      for (int j = 0; j < MV; ++j) wo[j] = trF[(si * C + r * MV + j) * QF + q];
      nlflux::F<FLUX>(wo, dd, fo, g);
      const int r2n = region_nbr(r, dd, side);
      if (r2n < 0) {
        for (int j = 0; j < MV; ++j) out[j] = side * fo[j];  // region boundary: interior trace
      } else {
        double wn[MV], fn[MV];
        for (int j = 0; j < MV; ++j) wn[j] = trF[((si ^ 1) * C + r2n * MV + j) * QF + q];
        nlflux::F<FLUX>(wn, dd, fn, g);
        const double a = alpha[region_face(r % 3, r / 3, dd, side)];
        for (int j = 0; j < MV; ++j) {
          const double fh = side > 0 ? 0.5 * (fo[j] + fn[j]) - 0.5 * a * (wn[j] - wo[j])
                                     : 0.5 * (fn[j] + fo[j]) - 0.5 * a * (wo[j] - wn[j]);
          out[j] = side * fh;
        }
      }
      const double s = 0.25 * lam[dd] * tb.wF[dd * QF + q];
      for (int j = 0; j < MV; ++j) H[(si * C + r * MV + j) * QF + q] = s * out[j];
    }
    __syncthreads();
    double* K2 = k2 + dd * 2 * C * NB * NB;  // [side][c][a][bo]
    if (dd == 0) {
      apply1d<NQ, NQ, 1, 1, NB>(H, Zo, tb.V1, tb.V1, NQ, 2 * C, 2 * C);   // [side][c][qt][by]
      __syncthreads();
      apply1d<NQ, NB, 1, 2, NB>(Zo, K2, tb.V1, tb.V1, NQ, 2 * C, 2 * C);  // [side][c][a][by]
    } else {
      apply1d<NQ, 1, NQ, 0, NB>(H, Zo, tb.V1, tb.V1, NQ, 2 * C, 2 * C);   // [side][c][qt][bx]
      __syncthreads();
      apply1d<NQ, 1, NB, 2, NB>(Zo, K2, tb.V1, tb.V1, NQ, 2 * C, 2 * C);  // [side][c][a][bx]
    }
    __syncthreads();
  }
  // ---- R = time term - source - volume + faces ----
  for (int i = threadIdx.x; i < 9 * D::BS; i += kThreads) {
    const int c = i / THT, k = i % THT;  // c = r MV + j
    const int a = k / THS, s2 = k % THS, by = s2 / NB, bx = s2 % NB;
    const double* w = Ws + c * THT;
    double acc = 0.0;
    for (int e = 0; e < NB; ++e) acc = fma(tb.Mt[a * NB + e], w[e * THS + s2], acc);
    acc = fma(-tb.em[a], Qs[c * THS + s2], acc);
    acc -= rv[i];
    // x faces: phi_bx(+-1) times the face term of (a, by); y faces: phi_by(+-1) times (a, bx)
    acc = fma(tb.ep1[bx], k2[((0 * C + c) * NB + a) * NB + by], acc);
    acc = fma(tb.em1[bx], k2[((1 * C + c) * NB + a) * NB + by], acc);
    acc = fma(tb.ep1[by], k2[((2 * C + c) * NB + a) * NB + bx], acc);
    acc = fma(tb.em1[by], k2[((3 * C + c) * NB + a) * NB + bx], acc);
    Rs[i] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// quasi-quadrature-free Jacobian (eqs. Jacproj, Jacobian2)
// ---------------------------------------------------------------------------------------
// Projected F' of region cell r into FA (point-major m x m matrices):
//   [F'_x (QP) | F'_y (QP) | own face f (QPf) x 4 | neighbour face f (QPf) x 4]
// scaled by -lam_d / 4 (volume) and +lam_d / 4 (faces), the factors of eq. Jacobian2.
template <typename T, int NB, int MV, int FLUX>
__device__ void project_cell(const NlDev& tb, int r, const double* Ws, const double* alpha,
                             T* FA, T* wp, T* b0, T* b1, const double* lam, double g) {
  using D = Dims<NB, MV>;
  constexpr int MM = D::MM, QP = D::QP, QPF = D::QPF, NP = D::NP, THT = D::THT;
  const T* PsiAtP = Tab<T>::PsiAtP(tb);
  const T* PsiAtFP = Tab<T>::PsiAtFP(tb);
  const T* P1 = Tab<T>::P1(tb);
  const T gT = (T)g;
  __shared__ T sclv[2], sclf[8];  // -lam_d / 4 per volume set, +lam_d / 4 per face set
  if (threadIdx.x < 2) sclv[threadIdx.x] = (T)(-0.25 * lam[threadIdx.x]);
  if (threadIdx.x < 8) sclf[threadIdx.x] = (T)(0.25 * lam[(threadIdx.x & 3) >> 1]);
  // volume: values at the projection points, F'_d there, three passes
  for (int i = threadIdx.x; i < MV * QP; i += kThreads) {
    const int j = i / QP, q = i % QP;
    wp[i] = dotcol<THT>(PsiAtP, QP, q, Ws + (r * MV + j) * THT);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < QP; q += kThreads) {
    T w[MV], J[MM];
    for (int j = 0; j < MV; ++j) w[j] = wp[j * QP + q];
    for (int dd = 0; dd < 2; ++dd) {
      nlflux::dF<FLUX>(w, dd, J, gT);
      for (int ij = 0; ij < MM; ++ij) b0[(dd * MM + ij) * QP + q] = J[ij];
    }
  }
  __syncthreads();
  proj_pass<NP, 3>(b0, b1, P1, 2 * MM, 0);
  __syncthreads();
  proj_pass<NP, 3>(b1, b0, P1, 2 * MM, 1);
  __syncthreads();
  proj_last<NP, 3, MM>(b0, FA, P1, 2, QP, 0, sclv);
  __syncthreads();
  // faces: the Rusanov flux Jacobian on both sides, at the face projection points
  for (int i = threadIdx.x; i < 4 * QPF; i += kThreads) {
    const int f = i / QPF, q = i % QPF;
    const int dd = f >> 1, si = f & 1, side = si ? -1 : 1;
    const T* to = PsiAtFP + (size_t)(dd * 2 + si) * THT * QPF;
    T wo[MV], Jo[MM];
    for (int j = 0; j < MV; ++j) wo[j] = dotcol<THT>(to, QPF, q, Ws + (r * MV + j) * THT);
    nlflux::dF<FLUX>(wo, dd, Jo, gT);
    const int r2 = region_nbr(r, dd, side);
    if (r2 < 0) {
      for (int ij = 0; ij < MM; ++ij) {
        b0[(f * MM + ij) * QPF + q] = side * Jo[ij];
        b0[((4 + f) * MM + ij) * QPF + q] = T(0);
      }
    } else {
      const T* tn = PsiAtFP + (size_t)(dd * 2 + (si ^ 1)) * THT * QPF;
      T wn[MV], Jn[MM];
      for (int j = 0; j < MV; ++j) wn[j] = dotcol<THT>(tn, QPF, q, Ws + (r2 * MV + j) * THT);
      nlflux::dF<FLUX>(wn, dd, Jn, gT);
      const T a = (T)alpha[region_face(r % 3, r / 3, dd, side)];
      // d F-hat / d w_L = (F'(w_L) + alpha I) / 2, d F-hat / d w_R = (F'(w_R) - alpha I) / 2,
      // times the outward sign of the face
      for (int i2 = 0; i2 < MV; ++i2)
        for (int j2 = 0; j2 < MV; ++j2) {
          const int ij = i2 * MV + j2;
          const T dg = i2 == j2 ? a : T(0);
          b0[(f * MM + ij) * QPF + q] = side > 0 ? T(0.5) * (Jo[ij] + dg) : T(-0.5) * (Jo[ij] - dg);
          b0[((4 + f) * MM + ij) * QPF + q] = side > 0 ? T(0.5) * (Jn[ij] - dg) : T(-0.5) * (Jn[ij] + dg);
        }
    }
  }
  __syncthreads();
  proj_pass<NP, 2>(b0, b1, P1, 8 * MM, 0);
  __syncthreads();
  proj_last<NP, 2, MM>(b1, FA, P1, 8, QPF, 2 * QP, sclf);
  __syncthreads();
}

// acc[g][ij] += sum over the list entries [e0, e1) of c * FA[g][off][ij]; the entries are
// fetched several at a time so that their memory latencies overlap
template <typename T, int CG, int MM, int FAS>
__device__ __forceinline__ void list_accumulate(const Ent<T>* __restrict__ ent, int e0, int e1,
                                                const T* FA, T (&acc)[CG][MM]) {
  constexpr int U = MM == 1 ? 8 : 1;  // wide (system) accumulators leave no registers for more
  for (int e = e0; e < e1; e += U) {
    Ent<T> en[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e + u < e1) en[u] = ent[e + u];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e + u >= e1) break;
      const T* v = FA + en[u].off * MM;
#pragma unroll
      for (int g = 0; g < CG; ++g)
#pragma unroll
        for (int ij = 0; ij < MM; ++ij) acc[g][ij] = fma(en[u].c, v[g * FAS + ij], acc[g][ij]);
    }
  }
}

// Assemble the diagonal blocks of cells r0 .. r0 + CG - 1 and their blocks towards the
// region neighbours from the merged lists (one pass over the lists for all CG cells).  In
// the tensor-core form a block (r, r2) with r2 eliminated after r is stored transposed.
template <typename T, int NB, int MV, bool TC>
__device__ void assemble_cells(const NlDev& tb, const NlPlan& plan, int r0, const T* FA,
                               T* slots) {
  using D = Dims<NB, MV>;
  constexpr int MM = D::MM, THT = D::THT, BP = D::BP, CG = D::CG, FAS = D::FAS;
  const Ent<T>* dent = Tab<T>::dent(tb);
  const T* Mt = Tab<T>::Mt(tb);
  for (int i = threadIdx.x; i < THT * THT; i += kThreads) {
    const int k = i / THT, l = i % THT;
    T acc[CG][MM];
#pragma unroll
    for (int g = 0; g < CG; ++g)
#pragma unroll
      for (int ij = 0; ij < MM; ++ij) acc[g][ij] = T(0);
    list_accumulate<T, CG, MM, FAS>(dent, tb.dptr[i], tb.dptr[i + 1], FA, acc);
    if (k % D::THS == l % D::THS) {
      const T mt = Mt[(k / D::THS) * NB + l / D::THS];
#pragma unroll
      for (int g = 0; g < CG; ++g)
#pragma unroll
        for (int j = 0; j < MV; ++j) acc[g][j * MV + j] += mt;
    }
#pragma unroll
    for (int g = 0; g < CG; ++g) {
      T* blk = slots + (size_t)plan.slot[(r0 + g) * 10] * BP * BP;
#pragma unroll
      for (int i2 = 0; i2 < MV; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < MV; ++j2) blk[bidx<TC, BP>(i2 * THT + k, j2 * THT + l)] = acc[g][i2 * MV + j2];
    }
  }
  // zero padding rows / columns of every block written here: the block GEMMs run over the
  // padded size, so padding must hold zeros whatever the scratch held before (the set of
  // padding positions is the same for a block and its transpose)
  if constexpr (BP > D::BS) {
    constexpr int BS = D::BS, NPAD = (BP - BS) * BP + BS * (BP - BS);
    for (int g = 0; g < CG; ++g) {
      const int r = r0 + g;
      for (int f = -1; f < 4; ++f) {
        const int r2 = f < 0 ? r : region_nbr(r, f >> 1, (f & 1) ? -1 : 1);
        if (r2 < 0) continue;
        T* blk = slots + (size_t)plan.slot[r * 9 + r2] * BP * BP;
        for (int i = threadIdx.x; i < NPAD; i += kThreads) {
          if (i < (BP - BS) * BP) {
            blk[bidx<TC, BP>(BS + i / BP, i % BP)] = T(0);
          } else {
            const int j = i - (BP - BS) * BP;
            blk[bidx<TC, BP>(j / (BP - BS), BS + j % (BP - BS))] = T(0);
          }
        }
      }
    }
  }
  for (int f = 0; f < 4; ++f) {
    const int dd = f >> 1, side = (f & 1) ? -1 : 1;
    const Ent<T>* oent = Tab<T>::oent(tb, f);
    const int* optr = tb.optr[f];
    for (int i = threadIdx.x; i < THT * THT; i += kThreads) {
      const int k = i / THT, l = i % THT;
      T acc[CG][MM];
#pragma unroll
      for (int g = 0; g < CG; ++g)
#pragma unroll
        for (int ij = 0; ij < MM; ++ij) acc[g][ij] = T(0);
      list_accumulate<T, CG, MM, FAS>(oent, optr[i], optr[i + 1], FA, acc);
#pragma unroll
      for (int g = 0; g < CG; ++g) {
        const int r = r0 + g, r2 = region_nbr(r, dd, side);
        if (r2 < 0) continue;
        T* blk = slots + (size_t)plan.slot[r * 9 + r2] * BP * BP;
        const bool tr = TC && plan.pos[r] < plan.pos[r2];
#pragma unroll
        for (int i2 = 0; i2 < MV; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < MV; ++j2)
            blk[bidx<TC, BP>(i2 * THT + k, j2 * THT + l, tr)] = acc[g][i2 * MV + j2];
      }
    }
  }
  if constexpr (TC) asm volatile("fence.proxy.async.global;" ::: "memory");  // read by bulk copies
  __syncthreads();
}

// The blocks of region cell r (one conserved variable, FP32) from its projected arrays FA,
// the same sums as assemble_cells but factorised: with k = (a_k, y_k, x_k) (time, y, x
// indices) and the triple products of eqs. Jacproj / Jacobian2 products of 1D factors
// (T0 = int phi phi phi, T1 = int phi' phi phi, traces phi(+-1)), each dimension's sum is
// taken once for all the others instead of per (k, l) pair:
//   Vx[pt,py,xk,xl] = sum_px T1[xk,xl,px] Fx[pt,py,px],  Wy likewise with T0 and Fy;
//   Hf[pt,ok,ol]    = sum_po T0[ok,ol,po] Ff[pt,po] for the own side of face f;
//   U[pt,yk,yl,xk,xl] = sum_py (T0[yk,yl,py] Vx + T1[yk,yl,py] Wy)[pt,py,xk,xl]
//                     + the faces' Hf times their trace pairs;
//   J[k,l] = sum_pt T0[ak,al,pt] U[pt,yk,yl,xk,xl] (+ the time term);
// and each neighbour block N_f[k,l] = tr(x or y of k) tr'(... of l) sum_pt T0[ak,al,pt]
// Hn_f[pt,ok,ol].  S: the buffers (Layout::SFN floats).  At Q4 this takes ~0.4 M FMAs per
// cell where the merged lists take ~1.5 M and one table load per FMA.
template <int NB, bool TC>
__device__ void assemble_cell_sf(const NlDev& tb, const NlPlan& plan, int r, const float* FA,
                                 float* S, float* slots) {
  using D = Dims<NB, 1>;
  constexpr int NP = D::NP, QP = D::QP, QPF = D::QPF, THS = D::THS, THT = D::THT;
  constexpr int BP = D::BP, BS = D::BS, NB2 = NB * NB, NB4 = NB2 * NB2, NP2 = NP * NP;
  const int tid = threadIdx.x;
  const float* T0 = tb.T0_f;
  const float* T1 = tb.T1_f;
  const float* ep = tb.ep1_f;
  const float* em = tb.em1_f;
  const float* Mt = tb.Mt_f;
  float* Vx = S;
  float* Wy = Vx + NP2 * NB2;
  float* U = Wy + NP2 * NB2;
  float* H = U + NP * NB4;
  float* K = H + 4 * NP * NB2;
  const float* Fx = FA;
  const float* Fy = FA + QP;
  const float* Ff = FA + 2 * QP;  // own side of face f at f QPF, the neighbour's at (4 + f) QPF
  for (int i = tid; i < NP2 * NB2; i += kThreads) {
    const int ptpy = i / NB2, kl = i - ptpy * NB2;
    const float* fx = Fx + ptpy * NP;
    const float* fy = Fy + ptpy * NP;
    const float* t1 = T1 + kl * NP;
    const float* t0 = T0 + kl * NP;
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      sx = fmaf(t1[p], fx[p], sx);
      sy = fmaf(t0[p], fy[p], sy);
    }
    Vx[i] = sx;
    Wy[i] = sy;
  }
  for (int i = tid; i < 4 * NP * NB2; i += kThreads) {
    const int fpt = i / NB2, kl = i - fpt * NB2;  // fpt = f NP + pt
    const int f = fpt / NP, pt = fpt - f * NP;
    const float* ff = Ff + f * QPF + pt * NP;
    const float* t0 = T0 + kl * NP;
    float h = 0.f;
#pragma unroll
    for (int p = 0; p < NP; ++p) h = fmaf(t0[p], ff[p], h);
    H[i] = h;
  }
  __syncthreads();
  for (int i = tid; i < NP * NB4; i += kThreads) {
    const int pt = i / NB4, rem = i - pt * NB4, ykl = rem / NB2, xkl = rem - ykl * NB2;
    const int yk = ykl / NB, yl = ykl - yk * NB, xk = xkl / NB, xl = xkl - xk * NB;
    const float* t0 = T0 + ykl * NP;
    const float* t1 = T1 + ykl * NP;
    const float* vx = Vx + pt * NP * NB2 + xkl;
    const float* wy = Wy + pt * NP * NB2 + xkl;
    float u = 0.f;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      u = fmaf(t0[p], vx[p * NB2], u);
      u = fmaf(t1[p], wy[p * NB2], u);
    }
    // own sides of the faces x+ (f 0), x- (1), y+ (2), y- (3): trace pairs of the normal index
    u = fmaf(ep[xk] * ep[xl], H[(0 * NP + pt) * NB2 + ykl], u);
    u = fmaf(em[xk] * em[xl], H[(1 * NP + pt) * NB2 + ykl], u);
    u = fmaf(ep[yk] * ep[yl], H[(2 * NP + pt) * NB2 + xkl], u);
    u = fmaf(em[yk] * em[yl], H[(3 * NP + pt) * NB2 + xkl], u);
    U[i] = u;
  }
  __syncthreads();
  {
    float* blk = slots + (size_t)plan.slot[r * 10] * BP * BP;
    for (int i = tid; i < THT * THT; i += kThreads) {
      const int k = i / THT, l = i - k * THT;
      const int ak = k / THS, sk = k - ak * THS, al = l / THS, sl = l - al * THS;
      const int yk = sk / NB, xk = sk - yk * NB, yl = sl / NB, xl = sl - yl * NB;
      const float* t0 = T0 + (ak * NB + al) * NP;
      const float* u = U + (yk * NB + yl) * NB2 + xk * NB + xl;
      float j = 0.f;
#pragma unroll
      for (int p = 0; p < NP; ++p) j = fmaf(t0[p], u[p * NB4], j);
      if (sk == sl) j += Mt[ak * NB + al];
      blk[bidx<TC, BP>(k, l)] = j;
    }
  }
  // the neighbour blocks, one face at a time (H and K reused)
  for (int f = 0; f < 4; ++f) {
    const int dd = f >> 1, si = f & 1;
    const int r2 = region_nbr(r, dd, si ? -1 : 1);
    if (r2 < 0) continue;  // (uniform over the block)
    __syncthreads();       // the previous face's K is consumed
    for (int i = tid; i < NP * NB2; i += kThreads) {
      const int pt = i / NB2, kl = i - pt * NB2;
      const float* ff = Ff + (4 + f) * QPF + pt * NP;
      const float* t0 = T0 + kl * NP;
      float h = 0.f;
#pragma unroll
      for (int p = 0; p < NP; ++p) h = fmaf(t0[p], ff[p], h);
      H[i] = h;
    }
    __syncthreads();
    for (int i = tid; i < NB4; i += kThreads) {
      const int akl = i / NB2, okl = i - akl * NB2;
      const float* t0 = T0 + akl * NP;
      float kk = 0.f;
#pragma unroll
      for (int p = 0; p < NP; ++p) kk = fmaf(t0[p], H[p * NB2 + okl], kk);
      K[i] = kk;
    }
    __syncthreads();
    // test function on this cell's side si of the face, trial function on the neighbour's
    // (opposite) side
    const float* trk = si ? em : ep;
    const float* trl = si ? ep : em;
    float* blk = slots + (size_t)plan.slot[r * 9 + r2] * BP * BP;
    const bool tr = TC && plan.pos[r] < plan.pos[r2];
    for (int i = tid; i < THT * THT; i += kThreads) {
      const int k = i / THT, l = i - k * THT;
      const int ak = k / THS, sk = k - ak * THS, al = l / THS, sl = l - al * THS;
      const int yk = sk / NB, xk = sk - yk * NB, yl = sl / NB, xl = sl - yl * NB;
      const int nk = dd == 0 ? xk : yk, nl = dd == 0 ? xl : yl;  // normal indices
      const int ok = dd == 0 ? yk : xk, ol = dd == 0 ? yl : xl;  // tangential indices
      blk[bidx<TC, BP>(k, l, tr)] = trk[nk] * trl[nl] * K[(ak * NB + al) * NB2 + ok * NB + ol];
    }
  }
  // zero padding rows / columns of every block written here (as in assemble_cells)
  if constexpr (BP > BS) {
    constexpr int NPAD = (BP - BS) * BP + BS * (BP - BS);
    for (int f = -1; f < 4; ++f) {
      const int r2 = f < 0 ? r : region_nbr(r, f >> 1, (f & 1) ? -1 : 1);
      if (r2 < 0) continue;
      float* blk = slots + (size_t)plan.slot[r * 9 + r2] * BP * BP;
      for (int i = tid; i < NPAD; i += kThreads) {
        if (i < (BP - BS) * BP) {
          blk[bidx<TC, BP>(BS + i / BP, i % BP)] = 0.f;
        } else {
          const int j = i - (BP - BS) * BP;
          blk[bidx<TC, BP>(j / (BP - BS), BS + j % (BP - BS))] = 0.f;
        }
      }
    }
  }
  if constexpr (TC) asm volatile("fence.proxy.async.global;" ::: "memory");  // read by bulk copies
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// dense block kernels of the elimination (T), all BP x BP row-major with zero padding.
// The 256 threads form a 16 x 16 grid; thread (ty, tx) owns rows ty + 16 a and columns
// tx + 16 b (a, b < RR) of a tile.
// ---------------------------------------------------------------------------------------
// Inverse of the leading BS x BS part of A (global) into S (shared, BP x BP, zero padding):
// Gauss-Jordan on a register-resident copy with implicit row pivoting (the pivot of column
// c is the largest remaining entry among the rows not yet used; no rows move), then the
// order is restored while writing S: with prow[c] the row that pivoted column c and rank its
// inverse permutation, inv[rank[i]][prow[j]] = R[i][j].
template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) { return __fdividef(1.0f, x); }  // ~2 ulp
template <>
__device__ __forceinline__ double recip<double>(double x) { return __drcp_rn(x); }

// Largest |v| over the candidates of the lanes in `mask` (valid != 0), ties to the lower
// row; the same result in every lane of the mask.  The magnitude's bit pattern orders like
// its value (v >= 0).
__device__ __forceinline__ int group_argmax(unsigned mask, float v, int row, bool valid, bool* zero) {
  const unsigned key = valid ? (__float_as_uint(v) | 0x80000000u) : 0u;
  const unsigned m = __reduce_max_sync(mask, key);
  const unsigned p = __reduce_min_sync(mask, key == m && valid ? (unsigned)row : 0xffffffffu);
  *zero = (m & 0x7fffffffu) == 0u;
  return (int)p;
}
__device__ __forceinline__ int group_argmax(unsigned mask, double v, int row, bool valid, bool* zero) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = valid ? ((unsigned)(b >> 32) | 0x80000000u) : 0u, lo = (unsigned)b;
  const unsigned mh = __reduce_max_sync(mask, hi);
  const bool h = valid && hi == mh;
  const unsigned ml = __reduce_max_sync(mask, h ? lo : 0u);
  const unsigned p = __reduce_min_sync(mask, h && lo == ml ? (unsigned)row : 0xffffffffu);
  *zero = (mh & 0x7fffffffu) == 0u && ml == 0u;
  return (int)p;
}

// x = a[k][j] for a block-uniform index k, without dynamic register indexing
template <typename T, int RR>
__device__ __forceinline__ void pick_row(const T (&a)[RR][RR], int k, T (&x)[RR]) {
  switch (k) {
    default:
#pragma unroll
      for (int j = 0; j < RR; ++j) x[j] = a[0][j];
      break;
#define RIDG_PICK_ROW(K) \
    case K:              \
      if constexpr (K < RR) { _Pragma("unroll") for (int j = 0; j < RR; ++j) x[j] = a[K][j]; } break;
    RIDG_PICK_ROW(1) RIDG_PICK_ROW(2) RIDG_PICK_ROW(3) RIDG_PICK_ROW(4) RIDG_PICK_ROW(5)
    RIDG_PICK_ROW(6) RIDG_PICK_ROW(7)
#undef RIDG_PICK_ROW
  }
}
// Pivot of one column, found by the half-warp that owns it (col = its entries in this
// thread's rows ty + 16 i, used = the rows that have pivoted): the column is published to
// cv, the pivot row to pv[0] and prow[c].
template <typename T, int BS, int RR>
__device__ __forceinline__ void gj_pivot(const T (&col)[RR], unsigned used, int ty,
                                         unsigned hmask, int c, T* cv, int* pv, int* prow,
                                         int* flags) {
  T best = T(0);
  int bi = 0;
  bool have = false;
#pragma unroll
  for (int i = 0; i < RR; ++i) {
    if ((used >> i) & 1u) continue;
    const T v = fabs(col[i]);
    if (!have || v > best) {
      best = v;
      bi = ty + 16 * i;
      have = true;
    }
  }
  bool zero = false;
  int p = group_argmax(hmask, best, bi, have, &zero);
  if (p >= BS) p = 0;  // unreachable: an unused row is always left
#pragma unroll
  for (int i = 0; i < RR; ++i) cv[ty + 16 * i] = col[i];
  if (ty == 0) {
    pv[0] = p;
    prow[c] = p;
    if (zero) atomicOr(flags, kFlagSingular);
  }
}

// Inverse of the leading BS x BS part of A (global) into S (BP x BP, zero padding; shared
// memory, or in the tensor-core form the block's own storage): Gauss-Jordan on a
// register-resident copy with implicit row pivoting (the pivot of column c is the largest
// remaining entry among the rows not yet used; no rows move), then the order is restored
// while writing S: with prow[c] the row that pivoted column c and rank its inverse
// permutation, inv[rank[i]][prow[j]] = R[i][j].
// Thread (tx, ty) = (tid / 16, tid % 16) owns rows ty + 16 i and columns tx + 16 j, so a
// column lives in one half-warp: that half-warp finds the pivot of its column and publishes
// the column, and each thread takes the pivot row from its own half-warp by shuffles -- one
// barrier per column.  Look-ahead: right after a step's barrier, the half-warp owning the
// next column updates that column alone, finds and publishes its pivot, and only then
// updates the rest of its tile, so the pivot search overlaps the elimination.  The columns
// run in blocks of 16 whose index cb is a compile-time constant (static register indexing).
template <typename T, int BS, int BP, int RR, bool TC = false>
__device__ void gj_inverse(const T* A, T* S, T* colv, T* rowp, int* prow, int* rank, int* flags) {
  static_assert(RR <= 8, "register tile up to 8 x 8");
  const int tid = threadIdx.x, tx = tid >> 4, ty = tid & 15;
  const int lane = tid & 31, half = lane & 16;
  const unsigned hmask = 0xFFFFu << half;
  T a[RR][RR];
#pragma unroll
  for (int i = 0; i < RR; ++i)
#pragma unroll
    for (int j = 0; j < RR; ++j) a[i][j] = A[bidx<TC, BP>(ty + 16 * i, tx + 16 * j)];
  unsigned used = 0u;  // bit i: row ty + 16 i has pivoted (or is padding)
#pragma unroll
  for (int i = 0; i < RR; ++i)
    if (ty + 16 * i >= BS) used |= 1u << i;
  int* pv = rank;      // pivot rows of the last two columns (rank is rebuilt at the end)
  if (tx == 0) {
    T col[RR];
#pragma unroll
    for (int i = 0; i < RR; ++i) col[i] = a[i][0];
    gj_pivot<T, BS, RR>(col, used, ty, hmask, 0, colv, pv, prow, flags);
  }
#pragma unroll
  for (int cb = 0; cb < RR; ++cb) {
    for (int cx = 0; cx < 16; ++cx) {
      const int c = cb * 16 + cx;
      if (c >= BS) break;
      const int buf = c & 1;
      const T* cv = colv + buf * BP;
      __syncthreads();  // column c and its pivot are published
      const int p = pv[buf];
      const T ipiv = recip(cv[p]);
      // the pivot row's entries in my columns, from the thread of my half-warp owning row p
      T mine[RR], prs[RR];
      pick_row(a, p >> 4, mine);
      const int src = half + (p & 15);
#pragma unroll
      for (int j = 0; j < RR; ++j) {
        const T v = __shfl_sync(0xffffffffu, mine[j], src);
        prs[j] = (j == cb && tx == cx) ? ipiv : v * ipiv;
      }
      if ((p & 15) == ty) used |= 1u << (p >> 4);
      // look-ahead: the owner of column c + 1 eliminates it first and publishes its pivot
      const int cn = c + 1;
      if (cn < BS && tx == (cn & 15)) {
        T col[RR];
        if ((cn >> 4) == cb) {
#pragma unroll
          for (int i = 0; i < RR; ++i) {
            const int ri = ty + 16 * i;
            col[i] = ri == p ? prs[cb] : fma(-cv[ri], prs[cb], a[i][cb]);
          }
        } else {
          const int jn = cb + 1 < RR ? cb + 1 : RR - 1;  // cb + 1 (a column of the next block)
#pragma unroll
          for (int i = 0; i < RR; ++i) {
            const int ri = ty + 16 * i;
            col[i] = ri == p ? prs[jn] : fma(-cv[ri], prs[jn], a[i][jn]);
          }
        }
        gj_pivot<T, BS, RR>(col, used, ty, hmask, cn, colv + (buf ^ 1) * BP, pv + (buf ^ 1), prow,
                            flags);
      }
#pragma unroll
      for (int i = 0; i < RR; ++i) {
        const int ri = ty + 16 * i;
        const T f = cv[ri];
        if (ri == p) {
#pragma unroll
          for (int j = 0; j < RR; ++j) a[i][j] = prs[j];
        } else {
#pragma unroll
          for (int j = 0; j < RR; ++j) a[i][j] = fma(-f, prs[j], a[i][j]);
          // column c: the elimination leaves -f_i / piv (1 / piv in the pivot row)
          if (tx == cx) a[i][cb] = -f * ipiv;
        }
      }
    }
  }
  __syncthreads();
  for (int c = tid; c < BS; c += kThreads) rank[prow[c]] = c;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RR; ++i) {
    const int ri = ty + 16 * i;
    if (ri >= BS) continue;
    const int rr = rank[ri];
#pragma unroll
    for (int j = 0; j < RR; ++j) {
      const int cj = tx + 16 * j;
      if (cj < BS) S[bidx<TC, BP>(rr, prow[cj])] = a[i][j];
    }
  }
  if constexpr (BP > BS) {
    for (int idx = tid; idx < (BP - BS) * BP; idx += kThreads) {
      S[bidx<TC, BP>(BS + idx / BP, idx % BP)] = T(0);                    // padding rows
      S[bidx<TC, BP>(idx / (BP - BS), BS + idx % (BP - BS))] = T(0);      // padding columns
    }
  }
  if constexpr (TC) asm volatile("fence.proxy.async.global;" ::: "memory");  // read by bulk copies
  __syncthreads();
}

// C = (overwrite ? 0 : C) - A B  (all global); staging double-buffered when NBUF == 2
template <typename T, int BP, int RR, int NBUF>
__device__ void gemm_sub(T* C, const T* A, const T* B, bool overwrite, T* sA, T* sB) {
  constexpr int NCH = BP / 16;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[RR][RR];
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) acc[a][b] = T(0);
  T pa[RR], pb[RR];
  auto gload = [&](int ch) {
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int idx = tid + kThreads * u;
      pa[u] = A[(size_t)(idx >> 4) * BP + ch * 16 + (idx & 15)];
      pb[u] = B[(size_t)(ch * 16 + idx / BP) * BP + idx % BP];
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int idx = tid + kThreads * u;
      sA[buf * BP * 17 + (idx >> 4) * 17 + (idx & 15)] = pa[u];
      sB[buf * 16 * BP + idx] = pb[u];
    }
  };
  gload(0);
  sstore(0);
  __syncthreads();
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = NBUF == 2 ? (ch & 1) : 0;
    if (NBUF == 2 && ch + 1 < NCH) gload(ch + 1);
    const T* a0 = sA + buf * BP * 17;
    const T* b0 = sB + buf * 16 * BP;
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      T av[RR], bv[RR];
#pragma unroll
      for (int a = 0; a < RR; ++a) av[a] = a0[(ty + 16 * a) * 17 + kk];
#pragma unroll
      for (int b = 0; b < RR; ++b) bv[b] = b0[kk * BP + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < RR; ++a)
#pragma unroll
        for (int b = 0; b < RR; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    if (NBUF == 2) {
      if (ch + 1 < NCH) sstore(buf ^ 1);
      __syncthreads();
    } else {
      __syncthreads();
      if (ch + 1 < NCH) {
        gload(ch + 1);
        sstore(0);
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) {
      T* c = C + (size_t)(ty + 16 * a) * BP + tx + 16 * b;
      *c = (overwrite ? T(0) : *c) - acc[a][b];
    }
}

// B = S B in place (S in shared memory, B in global memory)
template <typename T, int BP, int RR, int NBUF>
__device__ void gemm_left_inplace(const T* S, T* B, T* sB) {
  constexpr int NCH = BP / 16;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[RR][RR];
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) acc[a][b] = T(0);
  T pb[RR];
  auto gload = [&](int ch) {
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int idx = tid + kThreads * u;
      pb[u] = B[(size_t)(ch * 16 + idx / BP) * BP + idx % BP];
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int u = 0; u < RR; ++u) sB[buf * 16 * BP + tid + kThreads * u] = pb[u];
  };
  gload(0);
  sstore(0);
  __syncthreads();
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = NBUF == 2 ? (ch & 1) : 0;
    if (NBUF == 2 && ch + 1 < NCH) gload(ch + 1);
    const T* b0 = sB + buf * 16 * BP;
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      T av[RR], bv[RR];
#pragma unroll
      for (int a = 0; a < RR; ++a) av[a] = S[(ty + 16 * a) * BP + ch * 16 + kk];
#pragma unroll
      for (int b = 0; b < RR; ++b) bv[b] = b0[kk * BP + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < RR; ++a)
#pragma unroll
        for (int b = 0; b < RR; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    if (NBUF == 2) {
      if (ch + 1 < NCH) sstore(buf ^ 1);
      __syncthreads();
    } else {
      __syncthreads();
      if (ch + 1 < NCH) {
        gload(ch + 1);
        sstore(0);
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RR; ++b) B[(size_t)(ty + 16 * a) * BP + tx + 16 * b] = acc[a][b];
}

// y -= M x for the first BS rows (M global or shared, x and y shared).  Two threads per row,
// each summing half of the row with all of its vector loads issued back to back, so one
// memory round trip serves the whole block (BP <= 128, 256 threads).
template <typename T, int BS, int BP>
__device__ void matvec_sub(const T* M, const T* x, T* y) {
  constexpr int VW = sizeof(T) == 4 ? 4 : 2;  // elements per 16-byte vector
  constexpr int HALF = BP / 2;                // BP is a multiple of 16: HALF of VW
  constexpr int NV = HALF / VW;
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int r = threadIdx.x >> 1, h = threadIdx.x & 1;
  T s = T(0);
  if (r < BS) {
    const V* row = reinterpret_cast<const V*>(M + (size_t)r * BP + h * HALF);
    V v[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) v[u] = row[u];
    const T* xh = x + h * HALF;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      if constexpr (sizeof(T) == 4) {
        s = fma(v[u].x, xh[4 * u], s);
        s = fma(v[u].y, xh[4 * u + 1], s);
        s = fma(v[u].z, xh[4 * u + 2], s);
        s = fma(v[u].w, xh[4 * u + 3], s);
      } else {
        s = fma(v[u].x, xh[2 * u], s);
        s = fma(v[u].y, xh[2 * u + 1], s);
      }
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (r < BS && h == 0) y[r] -= s;
  __syncthreads();
}

// y -= M x for a block in the tensor-core storage (float): matvec_sub_c with M stored as
// itself (row r of M = storage row r: one 16-byte vector per 4-column chunk, two threads
// per row each taking half of the chunks), matvec_sub_t with M stored transposed (storage
// row j holds column j of M: TPC threads share one 4-row chunk of y, each summing every
// TPC-th column, then reduce by shuffles).
template <int BS, int BP>
__device__ void matvec_sub_c(const float* M, const float* x, float* y) {
  constexpr int NC = BP / 4, HC = NC / 2;  // BP is a multiple of 16: NC even
  const int r = threadIdx.x >> 1, h = threadIdx.x & 1;
  float s = 0.f;
  if (r < BS) {
    const float4* col = reinterpret_cast<const float4*>(M) + r;
    float4 v[HC];
#pragma unroll
    for (int u = 0; u < HC; ++u) v[u] = col[(h * HC + u) * BP];
    const float* xh = x + 4 * h * HC;
#pragma unroll
    for (int u = 0; u < HC; ++u) {
      s = fmaf(v[u].x, xh[4 * u], s);
      s = fmaf(v[u].y, xh[4 * u + 1], s);
      s = fmaf(v[u].z, xh[4 * u + 2], s);
      s = fmaf(v[u].w, xh[4 * u + 3], s);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (r < BS && h == 0) y[r] -= s;
  __syncthreads();
}

template <int BS, int BP>
__device__ void matvec_sub_t(const float* M, const float* x, float* y) {
  constexpr int NC = BP / 4;
  constexpr int TPC = NC <= 8 ? 32 : (NC <= 16 ? 16 : 8);  // threads per chunk, NC * TPC <= 256
  const int q = threadIdx.x / TPC, sub = threadIdx.x % TPC;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (q < NC) {
    const float4* ch = reinterpret_cast<const float4*>(M) + q * BP;
#pragma unroll 4
    for (int j = sub; j < BS; j += TPC) {
      const float4 v = ch[j];
      const float xj = x[j];
      acc.x = fmaf(v.x, xj, acc.x);
      acc.y = fmaf(v.y, xj, acc.y);
      acc.z = fmaf(v.z, xj, acc.z);
      acc.w = fmaf(v.w, xj, acc.w);
    }
  }
#pragma unroll
  for (int o = TPC / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
  }
  if (q < NC && sub == 0) {
    const int r = 4 * q;
    if (r < BS) y[r] -= acc.x;
    if (r + 1 < BS) y[r + 1] -= acc.y;
    if (r + 2 < BS) y[r + 2] -= acc.z;
    if (r + 3 < BS) y[r + 3] -= acc.w;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// tensor-core block products (TC form).  One thread issues the bulk copies of the K-slices
// and the MMAs; all threads then read the accumulator out of TMEM (thread <-> lane <-> row,
// the two warpgroups splitting the columns) and combine it with the destination block.
// Every wait is bounded: on a timeout the product reports failure (the CTA then stops).
// ---------------------------------------------------------------------------------------
struct TcCtx {
  uint32_t tmem;   // accumulator: 128 lanes x BP columns
  uint32_t ring;   // shared address of the stage ring
  uint32_t bar;    // full[kStages], empty[kStages], acc
  uint32_t fills;  // K-slices loaded so far (issuing thread only)
  uint32_t done;   // K-slices whose copies were waited for (issuing thread only)
  uint32_t gemms;  // products completed (every thread)
};

enum TcMode { kTcStore = 0, kTcNeg = 1, kTcSub = 2 };

__device__ __forceinline__ uint32_t tc_full(const TcCtx& tc, int st) { return tc.bar + 8u * st; }
__device__ __forceinline__ uint32_t tc_empty(const TcCtx& tc, int st) {
  return tc.bar + 8u * (kStages + st);
}
__device__ __forceinline__ uint32_t tc_acc(const TcCtx& tc) { return tc.bar + 8u * (2 * kStages); }

// D = Aop Bop^T over K = BP: Aop and Bop are BP x BP blocks in canonical storage (rows: M for
// Aop, N for Bop; columns: K).  Then C = D (kTcStore), C = -D (kTcNeg) or C -= D (kTcSub),
// with C in canonical storage whose rows are M.  Returns false (in every thread) if a wait
// timed out.
template <int BP>
__device__ bool tc_gemm(TcCtx& tc, const float* Aop, const float* Bop, float* C, int mode) {
  using TD = TcDims<BP>;
  constexpr int NS = TD::NS;
  const int tid = threadIdx.x;
  bool ok = true;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(128, BP);
    const uint32_t base = tc.fills;
    auto issue = [&](int sl) {
      const uint32_t g = tc.fills;
      const int st = (int)(g % kStages);
      if (g >= (uint32_t)kStages && !mbar_wait(tc_empty(tc, st), ((g / kStages) - 1u) & 1u)) return false;
      const uint32_t dst = tc.ring + st * TD::STAGE;
      mbar_expect_tx(tc_full(tc, st), 2u * TD::SL);
      bulk_load(dst, Aop + (size_t)sl * kKS * BP, TD::SL, tc_full(tc, st));
      bulk_load(dst + TD::SL + TD::PAD, Bop + (size_t)sl * kKS * BP, TD::SL, tc_full(tc, st));
      ++tc.fills;
      return true;
    };
    int next = 0;
    while (ok && next < NS && next < kStages) ok = issue(next++);
    for (int sl = 0; ok && sl < NS; ++sl) {
      const uint32_t g = base + sl;
      const int st = (int)(g % kStages);
      ok = mbar_wait(tc_full(tc, st), (g / kStages) & 1u);
      if (!ok) break;
      ++tc.done;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = tc.ring + st * TD::STAGE, b0 = a0 + TD::SL + TD::PAD;
#pragma unroll
      for (int kk = 0; kk < kKS / 8; ++kk)
        mma_tf32(tc.tmem, smem_desc(a0 + kk * 2u * BP * 16u, BP * 16u, 128u),
                 smem_desc(b0 + kk * 2u * BP * 16u, BP * 16u, 128u), idesc, (sl | kk) != 0);
      mma_commit(tc_empty(tc, st));
      // refill the stage of the previous slice (its MMAs are the oldest in flight)
      if (sl >= 1 && next < NS && next == sl - 1 + kStages) ok = issue(next++);
    }
    mma_commit(tc_acc(tc));  // arrives once every MMA issued so far is complete
  }
  const bool waited = mbar_wait_sleep(tc_acc(tc), tc.gemms & 1u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int warp = tid >> 5, lane = tid & 31, q = warp & 3, h = warp >> 2;
  const int row = 32 * q + lane;
  constexpr int HC = BP / 2, NG = HC / 8, GB = 4;  // column groups of 8, read GB at a time
#pragma unroll
  for (int g0 = 0; g0 < NG; g0 += GB) {
    uint32_t r[GB][8];
#pragma unroll
    for (int gi = 0; gi < GB; ++gi)
      if (g0 + gi < NG)
        tmem_ld8_nowait(tc.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * HC + 8 * (g0 + gi)), r[gi]);
    tmem_wait_ld();
    if (waited && row < BP) {
#pragma unroll
      for (int gi = 0; gi < GB; ++gi) {
        if (g0 + gi >= NG) break;
        const int c0 = h * HC + 8 * (g0 + gi);
        float4* p0 = reinterpret_cast<float4*>(C) + (c0 >> 2) * BP + row;
        float4* p1 = p0 + BP;
        float4 d0 = make_float4(__uint_as_float(r[gi][0]), __uint_as_float(r[gi][1]),
                                __uint_as_float(r[gi][2]), __uint_as_float(r[gi][3]));
        float4 d1 = make_float4(__uint_as_float(r[gi][4]), __uint_as_float(r[gi][5]),
                                __uint_as_float(r[gi][6]), __uint_as_float(r[gi][7]));
        if (mode == kTcSub) {
          const float4 o0 = *p0, o1 = *p1;
          d0 = make_float4(o0.x - d0.x, o0.y - d0.y, o0.z - d0.z, o0.w - d0.w);
          d1 = make_float4(o1.x - d1.x, o1.y - d1.y, o1.z - d1.z, o1.w - d1.w);
        } else if (mode == kTcNeg) {
          d0 = make_float4(-d0.x, -d0.y, -d0.z, -d0.w);
          d1 = make_float4(-d1.x, -d1.y, -d1.z, -d1.w);
        }
        *p0 = d0;
        *p1 = d1;
      }
    }
  }
  asm volatile("fence.proxy.async.global;" ::: "memory");  // C is read by later bulk copies
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  const bool all = __syncthreads_and((tid != 0 || ok) && waited) != 0;
  ++tc.gemms;
  return all;
}

// The issuing thread waits (bounded) for copies still in flight after a failed product, so
// that none lands in shared memory after the CTA has moved on or exited.
__device__ __forceinline__ void tc_drain(TcCtx& tc) {
  if (threadIdx.x == 0) {
    for (; tc.done < tc.fills; ++tc.done) {
      const uint32_t g = tc.done;
      (void)mbar_wait(tc_full(tc, (int)(g % kStages)), (g / kStages) & 1u);
    }
  }
  __syncthreads();
}

// Solve J x = b by block elimination in the plan's order; b in xs (9 x BP), x returned there.
template <typename T, int BS, int BP, int RR, int NBUF, bool KEEP>
__device__ void block_solve(T* slots, const NlPlan& plan, T* xs, T* S, T* sA, T* sB, T* colv,
                            T* rowp, int* prow, int* rank, int* flags) {
  const int tid = threadIdx.x;
  for (int t = 0; t < 9; ++t) {
    const int k = plan.order[t];
    T* Akk = slots + (size_t)plan.slot[k * 10] * BP * BP;
    gj_inverse<T, BS, BP, RR>(Akk, S, colv, rowp, prow, rank, flags);
    if (KEEP) {
      // keep the inverse in the (no longer needed) diagonal slot for later solves
      for (int i = tid; i < BP * BP; i += kThreads) Akk[i] = S[i];
    }
    // x_k <- S x_k (via a zeroed copy: y = x - S x computed as 0 - (-S) x is avoided by
    // writing the product straight into colv)
    T* xk = xs + k * BP;
    for (int i = tid; i < BP; i += kThreads) colv[i] = T(0);
    __syncthreads();
    matvec_sub<T, BS, BP>(S, xk, colv);  // colv = -S x_k
    for (int i = tid; i < BS; i += kThreads) xk[i] = -colv[i];
    __syncthreads();
    const int nn = plan.nn[t];
    for (int a = 0; a < nn; ++a) {
      const int j = plan.nbr[t][a];
      gemm_left_inplace<T, BP, RR, NBUF>(S, slots + (size_t)plan.slot[k * 9 + j] * BP * BP, sB);
    }
    __syncthreads();
    for (int a = 0; a < nn; ++a) {
      const int i = plan.nbr[t][a];
      const T* Aik = slots + (size_t)plan.slot[i * 9 + k] * BP * BP;
      matvec_sub<T, BS, BP>(Aik, xk, xs + i * BP);
      for (int b = 0; b < nn; ++b) {
        const int j = plan.nbr[t][b];
        gemm_sub<T, BP, RR, NBUF>(slots + (size_t)plan.slot[i * 9 + j] * BP * BP, Aik,
                                  slots + (size_t)plan.slot[k * 9 + j] * BP * BP,
                                  plan.first[t][a][b] != 0, sA, sB);
      }
    }
    __syncthreads();
  }
  for (int t = 8; t >= 0; --t) {
    const int k = plan.order[t];
    for (int a = 0; a < plan.nn[t]; ++a) {
      const int j = plan.nbr[t][a];
      matvec_sub<T, BS, BP>(slots + (size_t)plan.slot[k * 9 + j] * BP * BP, xs + j * BP, xs + k * BP);
    }
  }
}

// Solve J x = b again with the factors block_solve<KEEP = true> left in the slots (pivot
// inverses in the diagonal slots, A_ik below, U_kj above): block matvecs only.
template <typename T, int BS, int BP>
__device__ void stored_solve(const T* slots, const NlPlan& plan, T* xs, T* tmp) {
  const int tid = threadIdx.x;
  for (int t = 0; t < 9; ++t) {
    const int k = plan.order[t];
    T* xk = xs + k * BP;
    for (int i = tid; i < BP; i += kThreads) tmp[i] = T(0);
    __syncthreads();
    matvec_sub<T, BS, BP>(slots + (size_t)plan.slot[k * 10] * BP * BP, xk, tmp);  // -inv x_k
    for (int i = tid; i < BS; i += kThreads) xk[i] = -tmp[i];
    __syncthreads();
    for (int a = 0; a < plan.nn[t]; ++a) {
      const int i = plan.nbr[t][a];
      matvec_sub<T, BS, BP>(slots + (size_t)plan.slot[i * 9 + k] * BP * BP, xk, xs + i * BP);
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

// Tensor-core form of block_solve (T = float; the pivot inverses kept in the diagonal
// slots).  Storage: block (i, j) as itself when i is eliminated after j (or i == j), as its
// transpose when before -- so U_kj = A_kk^-1 A_kj is formed as U_kj^T = A_kj^T A_kk^-T and
// each Schur update A_ij -= A_ik U_kj as (A_ik)(U_kj^T)^T or, for a transposed A_ij, as
// (U_kj^T)(A_ik)^T: in every product both operands are read as stored.  Returns false if a
// tensor-core wait timed out.
template <int BS, int BP, int RR>
__device__ bool block_solve_tc(float* slots, const NlPlan& plan, float* xs, TcCtx& tc,
                               float* colv, float* rowp, int* prow, int* rank, int* flags) {
  const int tid = threadIdx.x;
  auto slot = [&](int i, int j) { return slots + (size_t)plan.slot[i * 9 + j] * BP * BP; };
  // the ring reuses shared memory the other phases wrote with ordinary stores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  bool ok = true;
  for (int t = 0; t < 9 && ok; ++t) {
    const int k = plan.order[t];
    float* Akk = slot(k, k);
    gj_inverse<float, BS, BP, RR, true>(Akk, Akk, colv, rowp, prow, rank, flags);
    float* xk = xs + k * BP;
    for (int i = tid; i < BP; i += kThreads) colv[i] = 0.f;
    __syncthreads();
    matvec_sub_c<BS, BP>(Akk, xk, colv);  // colv = -A_kk^-1 x_k
    for (int i = tid; i < BS; i += kThreads) xk[i] = -colv[i];
    __syncthreads();
    const int nn = plan.nn[t];
    for (int a = 0; a < nn && ok; ++a) {
      float* Akj = slot(k, plan.nbr[t][a]);
      ok = tc_gemm<BP>(tc, Akj, Akk, Akj, kTcStore);
    }
    for (int a = 0; a < nn && ok; ++a) {
      const int i = plan.nbr[t][a];
      const float* Aik = slot(i, k);
      matvec_sub_c<BS, BP>(Aik, xk, xs + i * BP);
      for (int b = 0; b < nn && ok; ++b) {
        const int j = plan.nbr[t][b];
        const float* Ukj = slot(k, j);
        const int mode = plan.first[t][a][b] ? kTcNeg : kTcSub;
        if (plan.pos[i] < plan.pos[j])
          ok = tc_gemm<BP>(tc, Ukj, Aik, slot(i, j), mode);
        else
          ok = tc_gemm<BP>(tc, Aik, Ukj, slot(i, j), mode);
      }
    }
  }
  if (!ok) return false;
  for (int t = 8; t >= 0; --t) {
    const int k = plan.order[t];
    for (int a = 0; a < plan.nn[t]; ++a) {
      const int j = plan.nbr[t][a];
      matvec_sub_t<BS, BP>(slot(k, j), xs + j * BP, xs + k * BP);
    }
  }
  return true;
}

// Solve J x = b again with the factors block_solve_tc left in the slots.
template <int BS, int BP>
__device__ void stored_solve_tc(const float* slots, const NlPlan& plan, float* xs, float* tmp) {
  const int tid = threadIdx.x;
  auto slot = [&](int i, int j) { return slots + (size_t)plan.slot[i * 9 + j] * BP * BP; };
  for (int t = 0; t < 9; ++t) {
    const int k = plan.order[t];
    float* xk = xs + k * BP;
    for (int i = tid; i < BP; i += kThreads) tmp[i] = 0.f;
    __syncthreads();
    matvec_sub_c<BS, BP>(slot(k, k), xk, tmp);  // -A_kk^-1 x_k
    for (int i = tid; i < BS; i += kThreads) xk[i] = -tmp[i];
    __syncthreads();
    for (int a = 0; a < plan.nn[t]; ++a) {
      const int i = plan.nbr[t][a];
      matvec_sub_c<BS, BP>(slot(i, k), xk, xs + i * BP);
    }
  }
  for (int t = 8; t >= 0; --t) {
    const int k = plan.order[t];
    for (int a = 0; a < plan.nn[t]; ++a) {
      const int j = plan.nbr[t][a];
      matvec_sub_t<BS, BP>(slot(k, j), xs + j * BP, xs + k * BP);
    }
  }
}

// ---------------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------------
// TMEM for the block products: 128 columns (>= BP for every degree), allocated once per CTA
__device__ __forceinline__ uint32_t tmem_alloc128(uint32_t* tslot) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *tslot;
}

__device__ __forceinline__ void tmem_free128(uint32_t tmem) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// Every region of one launch's degree, taken from its counter until it runs out.  The
// shared memory is laid out for this degree; with TC the CTA's TMEM columns (tmem) are given
// and the ring's barriers are initialised here (copies and products are all complete when
// this returns, so the next degree may reuse the same shared memory and TMEM).
template <typename T, int NB, int MV, int FLUX, bool TC, bool BATCH>
__device__ void newton_regions(const NewtonArgs& a, unsigned char* smem, uint32_t tmem) {
  static_assert(!TC || sizeof(T) == 4, "tensor-core block products are TF32 (T = float)");
  using D = Dims<NB, MV>;
  using L = Layout<T, NB, MV, TC>;
  double* Ws = (double*)(smem + L::oW);
  double* Qs = (double*)(smem + L::oQ);
  double* Rs = (double*)(smem + L::oR);
  double* alpha = (double*)(smem + L::oAl);
  double* red = (double*)(smem + L::oRed);
  T* xs = (T*)(smem + L::oX);
  T* colv = (T*)(smem + L::oCol);
  T* rowp = (T*)(smem + L::oRow);
  int* prow = (int*)(smem + L::oProw);
  int* rank = (int*)(smem + L::oRank);
  int* misc = (int*)(smem + L::oMisc);
  unsigned char* arena = smem + L::oArena;
  T* FA = (T*)arena;
  T* jw = (T*)(arena + L::oJW);
  T* jb0 = (T*)(arena + L::oJB0);
  T* jb1 = (T*)(arena + L::oJB1);
  T* S = (T*)arena;
  T* sA = (T*)(arena + L::oSA);
  T* sB = (T*)(arena + L::oSB);
  const int tid = threadIdx.x;
  T* slots = (T*)((char*)a.scratch + (size_t)blockIdx.x * a.scratch_per_cta);
  TcCtx tc{};
  if constexpr (TC) {
    // the ring's mbarriers (the TMEM accumulator is the caller's)
    tc.bar = smem_u32(smem + L::oBar);
    tc.ring = smem_u32(arena);
    if (tid == 0) {
      misc[1] = 0;
      for (int i = 0; i < 2 * kStages + 1; ++i) mbar_init(tc.bar + 8u * i, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tc.tmem = tmem;
  }

  for (;;) {
    if (tid == 0) misc[0] = atomicAdd(a.counter, 1);
    __syncthreads();
    const long long eg = misc[0];
    const bool stop = TC && misc[1] != 0;  // a tensor-core wait timed out
    __syncthreads();
    if (eg >= a.ncell || stop) break;
    // the region's instance: the handle's own mesh (its parameters read from the launch's
    // constant bank), or (batched launch) the last instance of the table whose first region
    // is <= eg, its parameters kept in shared memory
    RegionCtx* ctx = (RegionCtx*)(smem + L::oCtx);
    const double* Qg = a.Q;
    int nx = a.nx, ny = a.ny;
    long long e = eg;
    if constexpr (BATCH) {
      int lo = 0, hi = a.ninst - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.inst[mid].cell0 <= eg) lo = mid; else hi = mid - 1;
      }
      const NlInst& in = a.inst[lo];
      Qg = in.Q;
      nx = in.nx;
      ny = in.ny;
      e = eg - in.cell0;
      if (tid == 0) {
        ctx->e = e;
        ctx->lam[0] = in.lam[0];
        ctx->lam[1] = in.lam[1];
        ctx->W = in.W;
        ctx->stats = in.stats;
        ctx->itot = in.iters_total;
      }
    }
    const double* lam = BATCH ? ctx->lam : a.lam;
    const unsigned ue = (unsigned)e, uy = ue / (unsigned)nx;
    const int ix = (int)(ue - uy * (unsigned)nx), iy = (int)uy;
    for (int i = tid; i < 9 * MV * D::THS; i += kThreads) {
      const int r = i / (MV * D::THS), rem = i % (MV * D::THS);
      const long long c = (long long)((iy + r / 3 - 1 + ny) % ny) * nx + (ix + r % 3 - 1 + nx) % nx;
      Qs[i] = Qg[c * MV * D::THS + rem];
    }
    __syncthreads();
    int* const stats = BATCH ? ctx->stats : a.stats;  // after the barrier: ctx is written
    for (int i = tid; i < 9 * D::BS; i += kThreads) {
      const int r = i / D::BS, j = (i / D::THT) % MV, k = i % D::THT;
      Ws[i] = k < D::THS ? Qs[(r * MV + j) * D::THS + k] : 0.0;  // Q^n extended in time
    }
    __syncthreads();
    frozen_alpha<NB, MV, FLUX>(a.tb, Ws, alpha, (double*)arena, a.gamma);
    // FP64 form: Newton (a new Jacobian every iteration).  FP32 form: after a factorisation,
    // refinement sweeps reuse it with the FP64 residual while each contracts the update by
    // at least 10x (at most kSweeps per factorisation); max_iters caps the factorisations.
    // (TF32 block updates leave a coarser factorisation: more sweeps before a refactorisation)
    constexpr bool CHORD = sizeof(T) == 4;
    constexpr int kSweeps = TC ? 8 : 3;
    int it = 0, sweeps = 0;
    bool conv = false, bad = false, refactor = true;
    double dprev = 0.0;
    while (!conv && !bad) {
      if (refactor && it >= a.max_iters) break;
      residual<NB, MV, FLUX>(a.tb, Ws, Qs, Rs, alpha, (double*)arena, lam, a.gamma);
      if (refactor) {
        if constexpr (L::SF) {
          for (int r = 0; r < 9; ++r) {
            project_cell<T, NB, MV, FLUX>(a.tb, r, Ws, alpha, FA, jw, jb0, jb1, lam, a.gamma);
            assemble_cell_sf<NB, TC>(a.tb, a.plan, r, (const float*)FA, (float*)jw, (float*)slots);
          }
        } else {
          for (int r0 = 0; r0 < 9; r0 += D::CG) {
            for (int g = 0; g < D::CG; ++g)
              project_cell<T, NB, MV, FLUX>(a.tb, r0 + g, Ws, alpha, FA + g * D::FAS, jw, jb0,
                                            jb1, lam, a.gamma);
            assemble_cells<T, NB, MV, TC>(a.tb, a.plan, r0, FA, slots);
          }
        }
      }
      for (int i = tid; i < 9 * D::BP; i += kThreads) {
        const int r = i / D::BP, c = i % D::BP;
        xs[i] = c < D::BS ? (T)Rs[r * D::BS + c] : T(0);
      }
      __syncthreads();
      if constexpr (TC) {
        if (refactor) {
          if (!block_solve_tc<D::BS, D::BP, D::RR>(slots, a.plan, xs, tc, colv, rowp, prow, rank,
                                                    stats + 2)) {
            if (tid == 0) atomicOr(stats + 2, kFlagTimeout);
            misc[1] = 1;  // stop: the CTA's remaining regions are not solved
            break;
          }
        } else {
          stored_solve_tc<D::BS, D::BP>(slots, a.plan, xs, colv);
        }
      } else {
        if (refactor)
          block_solve<T, D::BS, D::BP, D::RR, L::NBUF, CHORD>(slots, a.plan, xs, S, sA, sB, colv,
                                                              rowp, prow, rank, stats + 2);
        else
          stored_solve<T, D::BS, D::BP>(slots, a.plan, xs, colv);
      }
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
      if (refactor) {
        ++it;
        sweeps = 0;
      } else {
        ++sweeps;
      }
      bad = nf > 0.0;
      conv = !bad && dn <= a.tol * fmax(1.0, wn);
      refactor = !CHORD || (sweeps > 0 && dn > 0.1 * dprev) || sweeps >= kSweeps;
      dprev = dn;
    }
    {
      double* W = BATCH ? ctx->W : a.W;
      const long long eo = BATCH ? ctx->e : e;
      for (int i = tid; i < D::BS; i += kThreads) W[eo * D::BS + i] = Ws[4 * D::BS + i];
    }
    if (tid == 0) {
      if (!conv) atomicAdd(&stats[0], 1);
      atomicMax(&stats[1], it);
      atomicAdd(&stats[7 + (it < 15 ? it : 15)], 1);  // histogram of iteration counts
      atomicAdd(BATCH ? ctx->itot : a.iters_total, (unsigned long long)it);
      if (bad) atomicOr(stats + 2, kFlagNonFinite);
    }
    __syncthreads();
  }
  if constexpr (TC) tc_drain(tc);
  __syncthreads();
}

template <typename T, int NB, int MV, int FLUX, bool TC, bool BATCH>
__global__ void __launch_bounds__(kThreads, (Layout<T, NB, MV, TC>::MINB)) newton_kernel(const NewtonArgs a) {
  using L = Layout<T, NB, MV, TC>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t tmem = 0;
  if constexpr (TC) tmem = tmem_alloc128((uint32_t*)(smem + L::oTmem));
  newton_regions<T, NB, MV, FLUX, TC, BATCH>(a, smem, tmem);
  if constexpr (TC) tmem_free128(tmem);
}

// The batched ensemble's Newton prediction in one launch: the degrees' region queues (each a
// NewtonArgs with its instance table and counter) in the given order, highest degree first;
// every CTA works through the first queue, then moves to the next as a queue runs out, so the
// lower degrees fill the tail of the higher ones.  Burgers (one conserved variable), degrees
// 1 to 4; shared memory is that of the largest degree.
template <typename T, bool TC>
struct MultiLayout {
  static constexpr size_t b2 = Layout<T, 2, 1, TC>::bytes, b3 = Layout<T, 3, 1, TC>::bytes,
                          b4 = Layout<T, 4, 1, TC>::bytes, b5 = Layout<T, 5, 1, TC>::bytes;
  static constexpr size_t bytes = cmax(cmax(b2, b3), cmax(b4, b5));
  // one CTA per SM: the four degrees' code in one kernel needs more than the 128 registers
  // a thread may hold at two CTAs of 256 threads (it spills 1 KB there)
  static constexpr int MINB = 1;
};

// (the degrees' arguments are read from device memory: four NewtonArgs are ~6 KB, more than
// one kernel parameter block should carry)
template <typename T, bool TC>
__global__ void __launch_bounds__(kThreads, (MultiLayout<T, TC>::MINB)) newton_multi_kernel(
    const NewtonMulti* __restrict__ m) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t tslot;
  uint32_t tmem = 0;
  if constexpr (TC) tmem = tmem_alloc128(&tslot);
  const int count = m->count;
  for (int g = 0; g < count; ++g) {
    const NewtonArgs& a = m->a[g];
    switch (m->nb[g]) {
      case 2: newton_regions<T, 2, 1, RIDG_FLUX_BURGERS, TC, true>(a, smem, tmem); break;
      case 3: newton_regions<T, 3, 1, RIDG_FLUX_BURGERS, TC, true>(a, smem, tmem); break;
      case 4: newton_regions<T, 4, 1, RIDG_FLUX_BURGERS, TC, true>(a, smem, tmem); break;
      case 5: newton_regions<T, 5, 1, RIDG_FLUX_BURGERS, TC, true>(a, smem, tmem); break;
      default: break;
    }
  }
  if constexpr (TC) tmem_free128(tmem);
}

// host: the same arguments in host memory (the counters to zero); dev: their device copy
template <typename T, bool TC>
cudaError_t launch_multi_typed(const NewtonMulti& host, const NewtonMulti* dev, int grid,
                               cudaStream_t s) {
  using ML = MultiLayout<T, TC>;
  static_assert(ML::bytes <= 232448, "Newton kernel shared memory above the per-CTA limit");
  cudaError_t e = cudaFuncSetAttribute(newton_multi_kernel<T, TC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ML::bytes);
  if (e != cudaSuccess) return e;
  for (int g = 0; g < host.count; ++g) {
    e = cudaMemsetAsync(host.a[g].counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  newton_multi_kernel<T, TC><<<grid, kThreads, ML::bytes, s>>>(dev);
  return cudaGetLastError();
}

template <typename T, bool TC>
int multi_ctas_per_sm() {
  return MultiLayout<T, TC>::MINB;
}

template <typename T, int NB, int MV, int FLUX, bool TC>
cudaError_t launch_one(const NewtonArgs& a, int grid, cudaStream_t s) {
  using L = Layout<T, NB, MV, TC>;
  static_assert(L::bytes <= 232448, "Newton kernel shared memory above the per-CTA limit");
  auto kern = a.ninst > 0 ? newton_kernel<T, NB, MV, FLUX, TC, true>
                          : newton_kernel<T, NB, MV, FLUX, TC, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, L::bytes, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int NB, int MV, int FLUX, bool TC>
int ctas_one() {
  using L = Layout<T, NB, MV, TC>;
  if (cudaFuncSetAttribute(newton_kernel<T, NB, MV, FLUX, TC, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, newton_kernel<T, NB, MV, FLUX, TC, false>,
                                                    kThreads, L::bytes) != cudaSuccess)
    return 0;
  // The occupancy calculator counts one CTA per SM for any kernel that uses tcgen05; the
  // tensor-core form still runs as many CTAs as its shared memory and registers allow
  // (MINB, at most 2 here), each holding 128 of the SM's 512 TMEM columns.
  return TC ? L::MINB : n;
}

// resident CTAs per SM of the Newton kernel for (nb, m, flux), 0 if unsupported
template <typename T, bool TC>
int ctas_per_sm(int nb, int m, int kind) {
  if (kind == RIDG_FLUX_BURGERS && m == 1) {
    switch (nb) {
      case 2: return ctas_one<T, 2, 1, RIDG_FLUX_BURGERS, TC>();
      case 3: return ctas_one<T, 3, 1, RIDG_FLUX_BURGERS, TC>();
      case 4: return ctas_one<T, 4, 1, RIDG_FLUX_BURGERS, TC>();
      case 5: return ctas_one<T, 5, 1, RIDG_FLUX_BURGERS, TC>();
      default: break;
    }
  } else if (kind == RIDG_FLUX_EULER && m == 4) {
    switch (nb) {
      case 2: return ctas_one<T, 2, 4, RIDG_FLUX_EULER, TC>();
      case 3: return ctas_one<T, 3, 4, RIDG_FLUX_EULER, TC>();
      default: break;
    }
  }
  return 0;
}

template <typename T, bool TC>
cudaError_t launch_typed(int nb, int m, int kind, const NewtonArgs& a, int grid, cudaStream_t s) {
  if (kind == RIDG_FLUX_BURGERS && m == 1) {
    switch (nb) {
      case 2: return launch_one<T, 2, 1, RIDG_FLUX_BURGERS, TC>(a, grid, s);
      case 3: return launch_one<T, 3, 1, RIDG_FLUX_BURGERS, TC>(a, grid, s);
      case 4: return launch_one<T, 4, 1, RIDG_FLUX_BURGERS, TC>(a, grid, s);
      case 5: return launch_one<T, 5, 1, RIDG_FLUX_BURGERS, TC>(a, grid, s);
      default: break;
    }
  } else if (kind == RIDG_FLUX_EULER && m == 4) {
    switch (nb) {
      case 2: return launch_one<T, 2, 4, RIDG_FLUX_EULER, TC>(a, grid, s);
      case 3: return launch_one<T, 3, 4, RIDG_FLUX_EULER, TC>(a, grid, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace newton
}  // namespace ridg
