// Mixed-precision linear prediction in 3D on the 5th-generation tensor cores (tcgen05 + TMA).
//
// What is computed: the time-mean prediction W-bar_e = P-bar X_e of every cell e (Sec. 2.2,
// eq. pred_full_system for a linear flux; X_e = the theta_S coefficients of the region cells
// upstream of e -- the upwind box, 2 x 2 x 2 of the 3 x 3 x 3 for a velocity with no zero
// component, the other cells' operator columns being zero -- and P-bar = the centre rows of
// the region operator that the correction of Sec. 2.3 needs), by the same split-operand
// refinement as the 2D path: the state as S balanced
// base-256 digits (exact in BF16) times one exponent, the operator rows likewise, digit
// products summed in FP32 per weight a + c' in TMEM and recombined with error-free sums.
//
// Tiles are 8 x 16 cells of one z-plane (M = 128).  The region offset (ox, oy, oz) is taken
// as in 2D -- x by one of the box's x-shifted TMA copies, y by the descriptor start -- and z
// by loading the plane z + oz.  Shared memory holds
//   the operator: the digits of every offset of the upwind box (at most 2 x 2 x 2 offsets;
//     98 KB at Q2 for the fused step operator's 64 padded rows with 3 slices, or for the 32
//     time-mean rows with 6), one stage per (oz, oy) row, bulk-copied once per CTA and kept
//     for all its tiles;
//   an A ring (2 to 8 slots, as many as fit): one digit of the box's input planes (per
//     plane one x-copy per x-offset, each 8-mode groups x 8 x 18 cells: 36.9 KB at Q2 for
//     two planes and two x-offsets), loaded by 4D TMA boxes of the ghost-padded digit planes.
// The MMA issuer runs digit a -> oz -> oy -> ox -> k-step; the epilogue writes the outputs
// as double-float pairs with a common exponent (or, for ridg_predict, FP64 rows), and the
// correction kernels apply them in double-float FP32 (state update FP64) and write the next
// step's digit planes.  Every
// wait is bounded (status bit on timeout).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "k_tc.cuh"
#include "ridg_internal.h"

namespace ridg {
namespace {

constexpr int kNAmax = 8;  // A slots (at most)
// warp 0: TMA producer, warp 1: MMA issuer, warps 2..17: epilogue (four per TMEM lane
// quadrant, each a quarter of the output columns)
constexpr int kEpiWarps = 16;
constexpr int kGemm3Threads = 32 * (2 + kEpiWarps);

struct Gemm3Layout {
  int P, brows, na, nst;
  uint32_t copy_bytes, z_bytes, a_bytes, b_bytes, b_off, bar_off, bytes;
};

// nop = padded output rows (32 or 64); ncx, ncy, ncz = offsets of the upwind box per
// dimension (an A slot holds one digit of the ncz input planes, each as ncx x-shifted
// copies; operator blocks per B stage, B stages = ncy ncz); the A ring takes the room that
// is left
__host__ __device__ inline Gemm3Layout gemm3_layout(int S, int thS, int nop, int ncx, int ncy,
                                                   int ncz, int na_cap = kNAmax) {
  Gemm3Layout l;
  l.P = ((thS + 15) / 16) * 2;
  l.brows = S * nop;
  l.copy_bytes = (uint32_t)l.P * kCopy * 16;
  l.z_bytes = ((uint32_t)ncx * l.copy_bytes + 1023u) & ~1023u;
  l.a_bytes = (uint32_t)ncz * l.z_bytes;
  l.b_bytes = (uint32_t)ncx * l.P * l.brows * 16;
  l.nst = ncy * ncz;
  const uint32_t btot = (uint32_t)l.nst * l.b_bytes;
  const uint32_t room = kSmemLimit - 1024u - btot;  // barriers and alignment slack
  int na = (int)(room / l.a_bytes);
  const int cap = na_cap > 0 && na_cap < kNAmax ? na_cap : kNAmax;
  l.na = na > cap ? cap : na;
  l.b_off = (uint32_t)l.na * l.a_bytes;
  l.bar_off = (l.b_off + btot + 63u) & ~63u;
  l.bytes = l.bar_off + 256;
  return l;
}

// float * 2^k as a double, by exponent arithmetic on the bits (exact; 0 stays 0)
__device__ __forceinline__ double f2d_scale(float f, int k) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e8 = (b >> 23) & 0xFF;
  if (e8 == 0) return 0.0;
  const int e11 = (int)e8 - 127 + 1023 + k;
  if (e11 <= 0) return 0.0;
  const uint32_t hiw = (b & 0x80000000u) | ((uint32_t)e11 << 20) | ((b & 0x7FFFFFu) >> 3);
  const uint32_t low = (b & 0x7u) << 29;
  return __hiloint2double((int)hiw, (int)low);
}

// NCXC = 2: the 2 x 2 x 2 upwind box, every offset loop unrolled; NCXC = 0: runtime counts.
template <int NB, int NCXC>
__global__ void __launch_bounds__(kGemm3Threads, 1) mixed3_gemm_kernel(
    const __grid_constant__ CUtensorMap dmap, const unsigned char* __restrict__ Bg,
    const float* __restrict__ rowmul, int S, int nout, int nop, float2* __restrict__ Y,
    double* __restrict__ W, int wstride, int wc0, int* __restrict__ exps,
    unsigned long long* __restrict__ maxbits, int nx, int ny, int nz, RegionBox box,
    int na_cap, int step, int wgmax, int* status) {
  constexpr int THS = NB * NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  constexpr int KSTEPS = P / 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_base_sh;
  // the upwind box: offsets lo + 0 .. cnt - 1 per dimension (cnt 1 or 2, at most 3 B stages)
  const int ox0 = box.lo[0], oy0 = box.lo[1], oz0 = box.lo[2];
  const int ncx = NCXC ? NCXC : box.cnt[0], ncy = NCXC ? NCXC : box.cnt[1],
            ncz = NCXC ? NCXC : box.cnt[2];
  const Gemm3Layout L = gemm3_layout(S, THS, nop, ncx, ncy, ncz, na_cap);
  const int NA = L.na;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty * nz;
  const int mytiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int tcols = S * nop;  // TMEM columns per stage (two stages; S nop <= 256)
  const uint32_t bar = smem_u32(smem + L.bar_off);
  const uint32_t afull0 = bar, afree0 = bar + 8u * kNAmax, bfull = bar + 16u * kNAmax,
                 tdone0 = bfull + 8u, tempty0 = tdone0 + 16u;
  const int sexp = exps[0];
  const bool f16 = exps[2] != 0;  // FP16 (else BF16) digit operands

  auto tile_origin = [&](int k, int& x0, int& y0, int& z0) {
    const int tile = blockIdx.x + k * gridDim.x;
    x0 = (tile % ntx) * kTX;
    y0 = ((tile / ntx) % nty) * kTY;
    z0 = tile / (ntx * nty);
  };

  if (tid == 0) {
    for (int i = 0; i < NA; ++i) {
      mbar_init(afull0 + 8u * i, 1);
      mbar_init(afree0 + 8u * i, 1);
    }
    mbar_init(bfull, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(tdone0 + 8u * i, 1);
      mbar_init(tempty0 + 8u * i, 32 * kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (blockIdx.x == 0 && step) {
      // rotate the running maximum: the correction that follows accumulates a fresh one
      maxbits[0] = maxbits[1];
      maxbits[1] = 0;
      exps[1] = sexp;  // exponent of this step's outputs, read by the correction
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: the operator once, then A digit planes in MMA order ----
      bool ok = true;
      if (mytiles > 0) {
        const uint32_t btot = (uint32_t)L.nst * L.b_bytes;
        mbar_expect_tx(bfull, btot);
        const uint32_t dst = smem_u32(smem + L.b_off);
        for (uint32_t off = 0; off < btot; off += 32768u)
          bulk_load(dst + off, Bg + off, min(32768u, btot - off), bfull);
      }
      int ia = 0;  // A items issued (one per tile and digit)
      for (int k = 0; k < mytiles && ok; ++k) {
        int x0, y0, z0;
        tile_origin(k, x0, y0, z0);
        for (int a = 0; a < S && ok; ++a, ++ia) {
          const int sl = ia % NA;
          if (ia >= NA && !mbar_wait_sleep(afree0 + 8u * sl, ((ia / NA) - 1) & 1)) { ok = false; break; }
          const uint32_t fa = afull0 + 8u * sl;
          // out-of-range boxes are zero-filled and counted
          mbar_expect_tx(fa, ncz * ncx * L.copy_bytes);
          const uint32_t dst = smem_u32(smem + sl * L.a_bytes);
          // plane jz, copy jx: x-offset ox0 + jx (padded column x0 + 1 + ox0 + jx, a multiple
          // of 8 elements), z-offset oz0 + jz (padded plane z0 + 1 + oz0 + jz)
          for (int jz = 0; jz < ncz; ++jz)
            for (int jx = 0; jx < ncx; ++jx)
              tma_load_4d(dst + jz * L.z_bytes + jx * L.copy_bytes, &dmap,
                          (x0 + 1 + ox0 + jx) * 8, y0, z0 + 1 + oz0 + jz, a * P, fa);
        }
      }
      if (!ok) atomicOr(status, kStatusTimeout);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t brows = (uint32_t)L.brows;
      const uint32_t copy16 = L.copy_bytes / 16;
      bool ok = true;
      if (mytiles > 0) {
        ok = mbar_wait(bfull, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      int ia = 0;
      for (int k = 0; k < mytiles && ok; ++k) {
        const int ts = k & 1;
        if (k >= 2 && !mbar_wait(tempty0 + 8u * ts, ((k - 2) >> 1) & 1)) { ok = false; break; }
        const uint32_t tst = tmem + (uint32_t)(ts * tcols);
        for (int a = 0; a < S && ok; ++a, ++ia) {
          const int sl = ia % NA;
          if (!mbar_wait(afull0 + 8u * sl, (ia / NA) & 1)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t idesc = idesc_digits(128, (S - a) * nop, f16);
          const uint32_t dcol = tst + (uint32_t)(a * nop);
#pragma unroll
          for (int jz = 0; jz < ncz; ++jz) {
            // A: LBO = plane stride inside a copy, SBO = one halo row of 8 cells (128 B)
            const uint64_t adesc0 =
                smem_desc(smem_u32(smem + sl * L.a_bytes + jz * L.z_bytes), kCopy * 16, 128);
#pragma unroll
            for (int jy = 0; jy < ncy; ++jy) {
              const uint64_t bdesc0 =
                  smem_desc(smem_u32(smem + L.b_off + (jz * ncy + jy) * L.b_bytes), brows * 16, 128);
              // y-offset oy0 + jy: the descriptor start moved by oy0 + jy + 1 halo rows
              const uint32_t yoff = (uint32_t)((oy0 + jy + 1) * kTX);
#pragma unroll
              for (int jx = 0; jx < (NCXC ? NCXC : ncx); ++jx) {
#pragma unroll
                for (int j = 0; j < KSTEPS; ++j) {
                  const uint32_t aoff = (uint32_t)jx * copy16 + (uint32_t)(2 * j * kCopy) + yoff;
                  const uint32_t boff = (uint32_t)(jx * P + 2 * j) * brows;
                  const uint32_t acc = (jz == 0 && a == 0 && jy == 0 && jx == 0 && j == 0) ? 0u : 1u;
                  mma_bf16(dcol, adesc0 + aoff, bdesc0 + boff, idesc, acc);
                }
              }
            }
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  afree0 + 8u * sl)
              : "memory");
        }
        if (ok)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  tdone0 + 8u * ts)
              : "memory");
      }
      if (!ok) atomicOr(status, kStatusTimeout);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 2..17, four per TMEM lane quadrant ----------------
    const int quad = warp & 3;  // (a warp reads the TMEM lanes of quadrant warp % 4)
    const int part = (warp - 2) >> 2;
    const int ncols = nop / 4;
    const int cell = quad * 32 + lane;
    const int ix = cell % kTX, iy = cell / kTX;
    const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
    const long long ncell = (long long)nx * ny * nz;
    for (int k = 0; k < mytiles; ++k) {
      const int ts = k & 1;
      if (!mbar_wait_sleep(tdone0 + 8u * ts, (k >> 1) & 1)) {
        if (lane == 0) atomicOr(status, kStatusTimeout);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int x0, y0, z0;
      tile_origin(k, x0, y0, z0);
      const int gx = x0 + ix, gy = y0 + iy;
      const long long e = ((long long)z0 * ny + gy) * nx + gx;
      const uint32_t tbase = lane_addr + (uint32_t)(ts * tcols);
#pragma unroll 1
      for (int cb = part * ncols; cb < (part + 1) * ncols; cb += 8) {
        if (cb >= nout) break;
        uint32_t raw[6][8];
#pragma unroll
        for (int t = 0; t < 6; ++t)
          if (t < S) tmem_ld8_nowait(tbase + (uint32_t)(t * nop + cb), raw[t]);
        tmem_wait_ld();
        float hi[8], lo[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          hi[c] = __uint_as_float(raw[0][c]);
          lo[c] = 0.f;
        }
        float w = 1.f;
#pragma unroll
        for (int t = 1; t < 6; ++t) {
          if (t < S) {
            w *= 1.f / 256.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              float s2, e2;
              two_sum(hi[c], __uint_as_float(raw[t][c]) * w, s2, e2);
              hi[c] = s2;
              lo[c] += e2;
            }
          }
        }
        if (gx < nx && gy < ny) {
          // (hi, lo) scaled to the common row exponent; value = (hi + lo) 2^(s + gmax - 16)
          if (W) {
            // (ridg_predict: FP64 straight into the cell's row of W, s = the planes' exponent)
            const int kw = sexp + wgmax - 16;
            double* wrow = W + e * wstride + wc0 + cb;
#pragma unroll
            for (int c = 0; c < 8; ++c)
              if (cb + c < nout) {
                const float m = rowmul[cb + c];
                wrow[c] = f2d_scale(hi[c] * m, kw) + f2d_scale(lo[c] * m, kw);
              }
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c)
              if (cb + c < nout) {
                const float m = rowmul[cb + c];
                Y[(long long)(cb + c) * ncell + e] = make_float2(hi[c] * m, lo[c] * m);
              }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(tempty0 + 8u * ts);
    }
  }
  // drain: no MMA may still write TMEM when it is released (bounded)
  if (tid == 0 && mytiles > 0) mbar_wait(tdone0 + 8u * ((mytiles - 1) & 1), ((mytiles - 1) >> 1) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------------------
// the correction of Sec. 2.3 from the double-float time means (value (hi + lo) 2^k, k = the
// outputs' exponent + gmax - 16): volume term sum_d nu_d (D along d) W-bar and upwind face
// values nu_d^+ tr_+(left) + nu_d^- tr_-(right), in double-float FP32; each face value is
// computed by both of its cells from the same traces in the same order (the same bits), the
// state update is FP64.  The kernel then writes the new state's digit planes (exponent from
// the previous maximum plus one bit of headroom, checked) and accumulates the new maximum.
// ---------------------------------------------------------------------------------------
// Unnormalised double-float values (s + e, |e| a few ulp of s at most) for the accumulations
// of the correction: a product costs 4 instructions and an accumulation 8, where the
// normalised pair arithmetic above costs 7 and 11; one normalisation at the end.
struct DFU {
  float s, e;
};

// c x, c = (ch, cl) and x = (xs, xe): ch xs exactly (product and FMA error), the cross terms
// ch xe + cl xs into the error word (cl xe is below the precision carried)
__device__ __forceinline__ DFU dfu_prod(float ch, float cl, float xs, float xe) {
  const float p = __fmul_rn(ch, xs);
  float e = __fmaf_rn(ch, xs, -p);
  e = __fmaf_rn(ch, xe, e);
  e = __fmaf_rn(cl, xs, e);
  return DFU{p, e};
}

// a += x: the leading words by an error-free sum, the error words added plainly
__device__ __forceinline__ void dfu_acc(DFU& a, DFU x) {
  float s, err;
  two_sum(a.s, x.s, s, err);
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(x.e, err));
}

// The update, one thread per cell.  Per direction d with velocity sign sg_d (the upwind
// side), per line t of the NB^2 lines of modes along d: the face values at the cell's two
// d-faces are the upwind traces nu_d tr(W-bar) -- of this cell and of its upstream neighbour
// (coalesced reads of the neighbour's time means; the neighbour's row was just read by the
// threads of that cell, so it is served by L2) -- computed by the same code from the same
// inputs in both cells of a face, so each face value has the same bits on both sides (exact
// conservation).  dQ = sum_d [(nu_d D[a][a-1]) W-bar(mode a-1 along d) + phi_a(+1) (s_a
// F(i - 1/2) - F(i + 1/2))], s_a = (-1)^a = phi_a(-1) / phi_a(+1), in double-float; then
// Q += dQ in FP64, the new state's digit rows (and ghost copies) and the running maximum.
// Degrees up to 2: a mode has at most one volume-term source per direction.
template <int NB, int S, int BT>
__global__ void __launch_bounds__(BT) mixed3_correct_kernel(
    double* __restrict__ Q, const float2* __restrict__ Y, int nx, int ny, int nz, CorrParams cp,
    int gmax, int* __restrict__ exps, unsigned long long* __restrict__ maxbits,
    uint4* __restrict__ planes, int* status) {
  static_assert(NB <= 3, "one volume-term source per mode and direction");
  constexpr int THS = NB * NB * NB, NT = NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  __shared__ unsigned long long shmax[8];
  // per-thread dQ accumulators (double-float), indexed by mode: in shared memory so that the
  // loops over lines stay rolled (a fully unrolled body stalls on instruction fetch); the
  // block size (64, 128 or 256 threads) is the autotuner's choice
  extern __shared__ float2 acc_sh[];
  float2* acc = acc_sh + threadIdx.x;  // mode s at acc[s * BT]
  const long long ncell = (long long)nx * ny * nz;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ys = exps[1];
  const int snext = exponent_above(maxbits[0]) + 1;
  unsigned long long mymax = 0;
  bool fits = true;
  if (e < ncell) {
    const unsigned ue = (unsigned)e, ur = ue / (unsigned)nx;
    const int ix = (int)(ue - ur * (unsigned)nx), iy = (int)(ur % (unsigned)ny), iz = (int)(ur / (unsigned)ny);
    for (int j = 0; j < THS; ++j) acc[j * BT] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int dd = 0; dd < 3; ++dd) {
      const double nu = cp.nu[dd];
      if (nu == 0.0) continue;  // no flux along d: no volume or face term
      const bool pos = nu > 0.0;
      // the upstream neighbour along d (periodic): i - 1 for nu > 0, i + 1 for nu < 0
      long long up;
      if (dd == 0) up = pos ? (ix == 0 ? e + (nx - 1) : e - 1) : (ix == nx - 1 ? e - (nx - 1) : e + 1);
      else if (dd == 1)
        up = pos ? (iy == 0 ? e + (long long)(ny - 1) * nx : e - nx)
                 : (iy == ny - 1 ? e - (long long)(ny - 1) * nx : e + nx);
      else
        up = pos ? (iz == 0 ? e + (long long)(nz - 1) * nx * ny : e - (long long)nx * ny)
                 : (iz == nz - 1 ? e - (long long)(nz - 1) * nx * ny : e + (long long)nx * ny);
      const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
      // upwind trace coefficients nu phi_b(+1) of the left cell (nu > 0) or nu phi_b(-1) =
      // nu (-1)^b phi_b(+1) of the right cell (nu < 0), as double-float pairs
      float ch[NB], cl[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        ch[b] = cp.tch[dd][b];
        cl[b] = cp.tcl[dd][b];
      }
      // the NB values of line t (modes base + b st) of a cell's time means sit at
      // Y[(base + b st) cells + e]; lines are walked as base = lo + hi, lo < st, hi in steps
      // of st NB (no divisions)
      const float2* Yo = Y + e;
      const float2* Yu = Y + up;
      const unsigned stn = (unsigned)st * (unsigned)ncell;
      // lines are walked with two cursors: the line computed (a) and the line whose values
      // are loaded, two ahead (b), so that two lines' loads are in flight
      int alo = 0, ahi = 0, blo = 0, bhi = 0;
      auto advance = [&](int& lo, int& hi) {
        if (++lo == st) {
          lo = 0;
          hi += st * NB;
        }
      };
      float2 co[NB], cu[NB], n1o[NB], n1u[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        co[b] = Yo[b * stn];
        cu[b] = Yu[b * stn];
      }
      advance(blo, bhi);
      {
        const unsigned off = (unsigned)(NT > 1 ? bhi + blo : 0) * (unsigned)ncell;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          n1o[b] = Yo[off + b * stn];
          n1u[b] = Yu[off + b * stn];
        }
      }
      advance(blo, bhi);
#pragma unroll 1
      for (int t = 0; t < NT; ++t) {
        const int base = ahi + alo;
        advance(alo, ahi);
        const unsigned noff = (unsigned)(t + 2 < NT ? bhi + blo : base) * (unsigned)ncell;
        if (t + 2 < NT) advance(blo, bhi);
        float2 no[NB], nu2[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          no[b] = Yo[noff + b * stn];
          nu2[b] = Yu[noff + b * stn];
        }
        // the face values nu tr(W-bar) of this cell and of the upstream neighbour (the same
        // code from the same inputs in both cells of a face: the same bits)
        DFU fo = dfu_prod(ch[0], cl[0], co[0].x, co[0].y);
        DFU fu = dfu_prod(ch[0], cl[0], cu[0].x, cu[0].y);
#pragma unroll
        for (int b = 1; b < NB; ++b) {
          dfu_acc(fo, dfu_prod(ch[b], cl[b], co[b].x, co[b].y));
          dfu_acc(fu, dfu_prod(ch[b], cl[b], cu[b].x, cu[b].y));
        }
        // F(i - 1/2), F(i + 1/2); mode a gets phi_a(+1) (s_a F(i - 1/2) - F(i + 1/2)), s_a =
        // (-1)^a: the even modes take dpos = F- - F+, the odd ones dneg = -(F- + F+)
        const DFU fm = pos ? fu : fo, fp = pos ? fo : fu;
        DFU dpos = fm, dneg = DFU{-fm.s, -fm.e};
        dfu_acc(dpos, DFU{-fp.s, -fp.e});
        dfu_acc(dneg, DFU{-fp.s, -fp.e});
#pragma unroll
        for (int a = 0; a < NB; ++a) {
          const float2 c = acc[(base + a * st) * BT];
          DFU v{c.x, c.y};
          if (a >= 1) dfu_acc(v, dfu_prod(cp.vdh[dd][a], cp.vdl[dd][a], co[a - 1].x, co[a - 1].y));
          const DFU df = (a & 1) ? dneg : dpos;
          // phi_0(+1) = 1 exactly
          dfu_acc(v, a == 0 ? df : dfu_prod(cp.eph[a], cp.epl[a], df.s, df.e));
          acc[(base + a * st) * BT] = make_float2(v.s, v.e);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          co[b] = n1o[b];
          cu[b] = n1u[b];
          n1o[b] = no[b];
          n1u[b] = nu2[b];
        }
      }
    }
    const int kfin = ys + gmax - 16;
    double* q = Q + e * THS;
    const long long pnx = nx + 2, pny = ny + 2;
    const long long plane = pnx * pny * (nz + 2);
    int px[2] = {ix + 1, -1}, py[2] = {iy + 1, -1}, pz[2] = {iz + 1, -1};
    if (ix == 0) px[1] = nx + 1;
    if (ix == nx - 1) px[1] = 0;
    if (iy == 0) py[1] = ny + 1;
    if (iy == ny - 1) py[1] = 0;
    if (iz == 0) pz[1] = nz + 1;
    if (iz == nz - 1) pz[1] = 0;
#pragma unroll 1
    for (int pg = 0; pg < P; ++pg) {
      double qn[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int sm = pg * 8 + j;
        if (sm < THS) {
          const float2 d = acc[sm * BT];
          double v = q[sm];
          v = v + f2d_scale(d.x, kfin);
          v = v + f2d_scale(d.y, kfin);
          q[sm] = v;
          qn[j] = v;
          const unsigned long long ab = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
          mymax = ab > mymax ? ab : mymax;
        } else {
          qn[j] = 0.0;
        }
      }
      uint4 rows[S];
      fits &= make_digit_rows<S>(qn, snext, rows, exps[2] != 0);
#pragma unroll
      for (int a = 0; a < S; ++a) {
        uint4* base = planes + (long long)(a * P + pg) * plane;
#pragma unroll
        for (int zi = 0; zi < 2; ++zi) {
          if (pz[zi] < 0) continue;
#pragma unroll
          for (int yi = 0; yi < 2; ++yi) {
            if (py[yi] < 0) continue;
#pragma unroll
            for (int xi = 0; xi < 2; ++xi) {
              if (px[xi] < 0) continue;
              base[((long long)pz[zi] * pny + py[yi]) * pnx + px[xi]] = rows[a];
            }
          }
        }
      }
    }
  }
  if (!fits) atomicOr(status, kStatusRange);
  const unsigned long long bm = block_max_bits(mymax, shmax);
  if (threadIdx.x == 0) {
    atomicMax(maxbits + 1, bm);
    if (blockIdx.x == 0) exps[0] = snext;
  }
}

// The update from the fused step operator's outputs, one thread per cell.  The prediction
// launch wrote, per cell, the volume term V_s = sum_d nu_d (D along d) W-bar (rows 0 ..
// theta_S - 1) and, per direction d and line t of the NB^2 lines of modes along d, the
// cell's upwind trace nu_d tr(W-bar) on its downstream d-face (rows theta_S + d NB^2 + t) --
// the face value of that face, read by both of its cells (the same bits on both sides:
// exact conservation).  dQ_s = V_s + sum_d phi_a(+1) (s_a F(i - 1/2) - F(i + 1/2)), a the
// mode's index along d, s_a = (-1)^a, F of a face = the trace of its upwind cell, in
// double-float.  Then the block updates its cells' state rows together (Q += dQ in FP64,
// read and written coalesced), and each thread writes its cell's digit rows (and ghost
// copies) and the running maximum, as in the kernel above.
template <int NB, int S, int BT>
__global__ void __launch_bounds__(BT) mixed3_fcorrect_kernel(
    double* __restrict__ Q, const float2* __restrict__ Y, int nx, int ny, int nz, CorrParams cp,
    int gmax, int* __restrict__ exps, unsigned long long* __restrict__ maxbits,
    uint4* __restrict__ planes, int* status) {
  constexpr int THS = NB * NB * NB, NT = NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  constexpr int PITCH = THS | 1;  // odd row pitch (8-byte words): conflict-free rows
  __shared__ unsigned long long shmax[8];
  // row c of the block's cell c: its dQ (double-float pairs) while the face terms are
  // summed, then its new state (FP64) in the same 8-byte words
  extern __shared__ float2 acc_sh[];
  float2* acc = acc_sh + threadIdx.x * PITCH;
  const long long ncell = (long long)nx * ny * nz;
  const long long e0 = (long long)blockIdx.x * BT;
  const int nblk = (int)min((long long)BT, ncell - e0);
  const long long e = e0 + threadIdx.x;
  const int ys = exps[1];
  const int snext = exponent_above(maxbits[0]) + 1;
  unsigned long long mymax = 0;
  bool fits = true;
  const unsigned ue = (unsigned)e, ur = ue / (unsigned)nx;
  const int ix = (int)(ue - ur * (unsigned)nx), iy = (int)(ur % (unsigned)ny), iz = (int)(ur / (unsigned)ny);
  if (e < ncell) {
    // the volume term (row 0, the cell mean's, is zero: the mean has no volume term)
#pragma unroll
    for (int j = 0; j < THS; ++j) acc[j] = Y[(unsigned)j * (unsigned)ncell + e];
    const float2* U = Y + (long long)THS * ncell;
#pragma unroll 1
    for (int dd = 0; dd < 3; ++dd) {
      const double nu = cp.nu[dd];
      if (nu == 0.0) continue;  // no flux along d: no volume or face term
      const bool pos = nu > 0.0;
      // the upstream neighbour along d (periodic): i - 1 for nu > 0, i + 1 for nu < 0
      long long up;
      if (dd == 0) up = pos ? (ix == 0 ? e + (nx - 1) : e - 1) : (ix == nx - 1 ? e - (nx - 1) : e + 1);
      else if (dd == 1)
        up = pos ? (iy == 0 ? e + (long long)(ny - 1) * nx : e - nx)
                 : (iy == ny - 1 ? e - (long long)(ny - 1) * nx : e + nx);
      else
        up = pos ? (iz == 0 ? e + (long long)(nz - 1) * nx * ny : e - (long long)nx * ny)
                 : (iz == nz - 1 ? e - (long long)(nz - 1) * nx * ny : e + (long long)nx * ny);
      const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
      const float2* Uo = U + (long long)dd * NT * ncell + e;   // this cell's traces
      const float2* Uu = U + (long long)dd * NT * ncell + up;  // the upstream neighbour's
      // the direction's 2 NB^2 traces, all loads in flight at once
      float2 to[NT], tu[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        to[t] = Uo[(unsigned)t * (unsigned)ncell];
        tu[t] = Uu[(unsigned)t * (unsigned)ncell];
      }
      // line t holds the modes base + a st; base walked as lo + hi (lo < st, hi in steps of
      // st NB), no divisions
      int lo = 0, hi = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int base = hi + lo;
        if (++lo == st) {
          lo = 0;
          hi += st * NB;
        }
        // F(i - 1/2) (the upstream cell's trace for nu > 0, this cell's for nu < 0) and
        // F(i + 1/2); even modes take dpos = F- - F+, odd ones dneg = -(F- + F+)
        const DFU fo{to[t].x, to[t].y}, fu{tu[t].x, tu[t].y};
        const DFU fm = pos ? fu : fo, fp = pos ? fo : fu;
        DFU dpos = fm, dneg = DFU{-fm.s, -fm.e};
        dfu_acc(dpos, DFU{-fp.s, -fp.e});
        dfu_acc(dneg, DFU{-fp.s, -fp.e});
#pragma unroll
        for (int a = 0; a < NB; ++a) {
          const float2 c = acc[base + a * st];
          DFU v{c.x, c.y};
          const DFU df = (a & 1) ? dneg : dpos;
          // phi_0(+1) = 1 exactly
          dfu_acc(v, a == 0 ? df : dfu_prod(cp.eph[a], cp.epl[a], df.s, df.e));
          acc[base + a * st] = make_float2(v.s, v.e);
        }
      }
    }
  }
  __syncthreads();
  // Q += dQ over the block's rows, element i = (cell i / THS, mode i % THS): coalesced
  const int kfin = ys + gmax - 16;
  double* sq = (double*)acc_sh;
  // (eight elements per thread at a time: their loads are in flight together)
  const int nel = nblk * THS;
  double* const Qb = Q + e0 * THS;
#pragma unroll 1
  for (int i0 = threadIdx.x; i0 < nel; i0 += 8 * BT) {
    double qv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * BT;
      qv[u] = i < nel ? Qb[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * BT;
      if (i < nel) {
        const int c = i / THS, k = c * PITCH + (i - c * THS);
        const float2 d = acc_sh[k];
        double v = qv[u];
        v = v + f2d_scale(d.x, kfin);
        v = v + f2d_scale(d.y, kfin);
        Qb[i] = v;
        sq[k] = v;
        const unsigned long long ab = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
        mymax = ab > mymax ? ab : mymax;
      }
    }
  }
  __syncthreads();
  if (e < ncell) {
    const double* q = sq + threadIdx.x * PITCH;
    const long long pnx = nx + 2, pny = ny + 2;
    const long long plane = pnx * pny * (nz + 2);
    const long long own = ((long long)(iz + 1) * pny + (iy + 1)) * pnx + (ix + 1);
    // a boundary cell also writes its periodic ghost copies
    const bool ghost = ix == 0 || ix == nx - 1 || iy == 0 || iy == ny - 1 || iz == 0 || iz == nz - 1;
#pragma unroll 1
    for (int pg = 0; pg < P; ++pg) {
      double qn[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) qn[j] = pg * 8 + j < THS ? q[pg * 8 + j] : 0.0;
      uint4 rows[S];
      fits &= make_digit_rows<S>(qn, snext, rows, exps[2] != 0);
#pragma unroll
      for (int a = 0; a < S; ++a) planes[(long long)(a * P + pg) * plane + own] = rows[a];
      if (ghost) {
        int px[2] = {ix + 1, -1}, py[2] = {iy + 1, -1}, pz[2] = {iz + 1, -1};
        if (ix == 0) px[1] = nx + 1;
        if (ix == nx - 1) px[1] = 0;
        if (iy == 0) py[1] = ny + 1;
        if (iy == ny - 1) py[1] = 0;
        if (iz == 0) pz[1] = nz + 1;
        if (iz == nz - 1) pz[1] = 0;
#pragma unroll 1
        for (int g = 1; g < 8; ++g) {
          const int zz = pz[g >> 2], yy = py[(g >> 1) & 1], xx = px[g & 1];
          if (zz < 0 || yy < 0 || xx < 0) continue;
          const long long o = ((long long)zz * pny + yy) * pnx + xx;
#pragma unroll
          for (int a = 0; a < S; ++a) planes[(long long)(a * P + pg) * plane + o] = rows[a];
        }
      }
    }
  }
  if (!fits) atomicOr(status, kStatusRange);
  const unsigned long long bm = block_max_bits(mymax, shmax);
  if (threadIdx.x == 0) {
    atomicMax(maxbits + 1, bm);
    if (blockIdx.x == 0) exps[0] = snext;
  }
}

// ---------------------------------------------------------------------------------------
// digit planes of the 3D state: plane (a * P + p), padded (z + 1, y + 1, x + 1), one thread
// per (cell, 8-mode group); the cell's periodic ghost copies are written too
// ---------------------------------------------------------------------------------------
template <int NB, int S>
__global__ void __launch_bounds__(128) state_digits3_kernel(const double* __restrict__ Q, int nx,
                                                            int ny, int nz,
                                                            const unsigned long long* maxbits,
                                                            int* exps, uint4* __restrict__ planes,
                                                            int* status) {
  constexpr int THS = NB * NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  const long long ncell = (long long)nx * ny * nz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = exponent_above(maxbits[1]) + 1;
  if (i == 0) exps[0] = s;
  if (i >= ncell * P) return;
  const long long e = i / P;
  const int p = (int)(i % P);
  const unsigned ue = (unsigned)e, ur = ue / (unsigned)nx;
  const int ix = (int)(ue - ur * (unsigned)nx), iy = (int)(ur % (unsigned)ny), iz = (int)(ur / (unsigned)ny);
  double v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = (p * 8 + j < THS) ? Q[e * THS + p * 8 + j] : 0.0;
  uint4 rows[S];
  if (!make_digit_rows<S>(v, s, rows, exps[2] != 0)) atomicOr(status, kStatusRange);
  const long long pnx = nx + 2, pny = ny + 2;
  const long long plane = pnx * pny * (nz + 2);
  int px[2] = {ix + 1, -1}, py[2] = {iy + 1, -1}, pz[2] = {iz + 1, -1};
  if (ix == 0) px[1] = nx + 1;
  if (ix == nx - 1) px[1] = 0;
  if (iy == 0) py[1] = ny + 1;
  if (iy == ny - 1) py[1] = 0;
  if (iz == 0) pz[1] = nz + 1;
  if (iz == nz - 1) pz[1] = 0;
#pragma unroll
  for (int a = 0; a < S; ++a) {
    uint4* base = planes + (long long)(a * P + p) * plane;
#pragma unroll
    for (int zi = 0; zi < 2; ++zi) {
      if (pz[zi] < 0) continue;
#pragma unroll
      for (int yi = 0; yi < 2; ++yi) {
        if (py[yi] < 0) continue;
#pragma unroll
        for (int xi = 0; xi < 2; ++xi) {
          if (px[xi] < 0) continue;
          base[((long long)pz[zi] * pny + py[yi]) * pnx + px[xi]] = rows[a];
        }
      }
    }
  }
}

// ridg_predict's outputs: W[e * wstride + c0 + c] = (hi + lo) 2^(s + gmax - 16) in FP64, s the
// planes' exponent (the launch that produced Y left the step's bookkeeping alone)
// (a tile of 32 cells x nout outputs through shared memory: Y read along the cells, W
// written along each cell's row)
__global__ void __launch_bounds__(256) mixed3_to_w_kernel(const float2* __restrict__ Y,
                                                          long long ncell, int nout, int c0,
                                                          int wstride, const int* __restrict__ exps,
                                                          int gmax, double* __restrict__ W) {
  constexpr int TPITCH = 33;  // odd: conflict-free reads along a cell's row
  __shared__ double tile[64 * TPITCH];
  const long long e0 = (long long)blockIdx.x * 32;
  const int nc = (int)min(32LL, ncell - e0);
  const int j = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int k = exps[0] + gmax - 16;
  if (j < nc)
    for (int c = r; c < nout; c += 8) {
      const float2 y = Y[(long long)c * ncell + e0 + j];
      tile[c * TPITCH + j] = f2d_scale(y.x, k) + f2d_scale(y.y, k);
    }
  __syncthreads();
  for (int f = threadIdx.x; f < nc * nout; f += 256) {
    const int jj = f / nout, c = f - jj * nout;
    W[(e0 + jj) * wstride + c0 + c] = tile[c * TPITCH + jj];
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
cudaError_t launch_mixed3_to_w(const Grid& g, int nout, int c0, int wstride, const void* Y,
                               int gmax, const MixedState& ms, double* W, cudaStream_t s) {
  if (nout < 1 || nout > 64) return cudaErrorInvalidValue;
  mixed3_to_w_kernel<<<(unsigned)((g.ncell + 31) / 32), 256, 0, s>>>((const float2*)Y, g.ncell,
                                                                    nout, c0, wstride, ms.exps,
                                                                    gmax, W);
  return cudaGetLastError();
}

bool mixed3_supported(int nb, int slices) {
  if (nb < 2 || nb > 3 || slices < 2 || slices > 6) return false;
  const Gemm3Layout l = gemm3_layout(slices, nb * nb * nb, 32, 2, 2, 2);  // widest upwind box
  return l.na >= 2 && l.bytes <= kSmemLimit;
}

int mixed3_fused_nout(int nb) { return nb * nb * nb + 3 * nb * nb; }

bool mixed3_fused_fits(int nb, int slices) {
  if (!mixed3_supported(nb, slices)) return false;
  const int nout = mixed3_fused_nout(nb), nop = nout <= 32 ? 32 : 64;
  if (nout > 64 || slices * nop > 256) return false;  // two TMEM stages, MMA N <= 256
  const Gemm3Layout l = gemm3_layout(slices, nb * nb * nb, nop, 2, 2, 2);
  return l.na >= 2 && l.bytes <= kSmemLimit;
}

size_t mixed3_plane_bytes(const Grid& g, int nb, int slices) {
  const int thS = nb * nb * nb, P = ((thS + 15) / 16) * 2;
  return (size_t)(g.n[0] + 2) * (g.n[1] + 2) * (g.n[2] + 2) * slices * P * 16;
}

int mixed3_make_map(const Grid& g, int nb, int slices, void* planes, void* map_out) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return RIDG_ECUDA;
  const int thS = nb * nb * nb, P = ((thS + 15) / 16) * 2;
  const cuuint64_t px = g.n[0] + 2, py = g.n[1] + 2, pz = g.n[2] + 2;
  // dims (fastest first): padded x times 8 modes (BF16), padded y, padded z, digit x group
  cuuint64_t dims[4] = {px * 8, py, pz, (cuuint64_t)slices * P};
  cuuint64_t strides[3] = {px * 16, px * py * 16, px * py * pz * 16};
  cuuint32_t box[4] = {(cuuint32_t)kTX * 8, (cuuint32_t)kHY, 1u, (cuuint32_t)P};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = ((EncodeFn)fn)((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, planes,
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RIDG_OK : RIDG_ECUDA;
}

template <int NB>
static cudaError_t launch_gemm3_t(const Grid& g, const MixedOp& op, MixedState& ms, void* Y,
                                  double* W, int wstride, int wc0, int slots, cudaStream_t s,
                                  bool step) {
  if (op.npad != 32 && op.npad != 64) return cudaErrorInvalidValue;
  if (op.slices * op.npad > 256 || op.nout > op.npad) return cudaErrorInvalidValue;
  const Gemm3Layout L = gemm3_layout(op.slices, NB * NB * NB, op.npad, g.box.cnt[0], g.box.cnt[1],
                                     g.box.cnt[2], slots);
  if (L.na < 2 || L.bytes > kSmemLimit) return cudaErrorInvalidValue;
  // one CTA per SM: each allocates all 512 TMEM columns, so a second CTA on the SM would
  // only wait for them -- ask for more than half the shared memory
  const uint32_t smem = std::max<uint32_t>(L.bytes, 117u * 1024u);
  const bool box222 = g.box.cnt[0] == 2 && g.box.cnt[1] == 2 && g.box.cnt[2] == 2;
  auto kern = box222 ? mixed3_gemm_kernel<NB, 2> : mixed3_gemm_kernel<NB, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = ((g.n[0] + kTX - 1) / kTX) * ((g.n[1] + kTY - 1) / kTY) * g.n[2];
  const int grid = std::min(ntiles, sms);
  kern<<<grid, kGemm3Threads, smem, s>>>(*(const CUtensorMap*)ms.map,
                                        (const unsigned char*)op.b_slices, op.row_mul, op.slices,
                                        op.nout, op.npad, (float2*)Y, W, wstride, wc0, ms.exps,
                                        ms.maxbits, g.n[0], g.n[1], g.n[2], g.box, slots,
                                        step ? 1 : 0, op.gmax, ms.status);
  return cudaGetLastError();
}

int mixed3_gemm_slots(int nb, int slices, int npad, const RegionBox& box, int cap) {
  const Gemm3Layout L =
      gemm3_layout(slices, nb * nb * nb, npad, box.cnt[0], box.cnt[1], box.cnt[2], cap);
  return L.na;
}

cudaError_t launch_mixed3_gemm(const Grid& g, int nb, const MixedOp& op, MixedState& ms, void* Y,
                               int slots, cudaStream_t s, bool step) {
  if (g.dim != 3 || g.box.n < 1 || g.box.n > 8 || op.K != g.box.n * nb * nb * nb)
    return cudaErrorInvalidValue;
  switch (nb) {
    case 2: return launch_gemm3_t<2>(g, op, ms, Y, nullptr, 0, 0, slots, s, step);
    case 3: return launch_gemm3_t<3>(g, op, ms, Y, nullptr, 0, 0, slots, s, step);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mixed3_predict(const Grid& g, int nb, const MixedOp& op, MixedState& ms,
                                  double* W, int wstride, int c0, int slots, cudaStream_t s) {
  if (g.dim != 3 || g.box.n < 1 || g.box.n > 8 || op.K != g.box.n * nb * nb * nb || !W ||
      c0 < 0 || c0 + op.nout > wstride)
    return cudaErrorInvalidValue;
  switch (nb) {
    case 2: return launch_gemm3_t<2>(g, op, ms, nullptr, W, wstride, c0, slots, s, false);
    case 3: return launch_gemm3_t<3>(g, op, ms, nullptr, W, wstride, c0, slots, s, false);
    default: return cudaErrorInvalidValue;
  }
}

template <int NB, int S>
static cudaError_t launch_correct3_t(const Grid& g, double* Q, const void* Y, int gmax,
                                     const CorrParams& cp, MixedState& ms, int block, bool fused,
                                     cudaStream_t s) {
  // the kernels index the outputs with 32-bit offsets (row x cells)
  if ((long long)g.ncell * mixed3_fused_nout(NB) >= (1LL << 32)) return cudaErrorInvalidValue;
  if (block != 64 && block != 128 && block != 256) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((g.ncell + block - 1) / block);
  // (the fused form keeps its rows at an odd pitch)
  constexpr int THS = NB * NB * NB;
  const size_t smem = (size_t)block * (fused ? (THS | 1) : THS) * sizeof(float2);
  auto kern = fused ? (block == 64    ? mixed3_fcorrect_kernel<NB, S, 64>
                       : block == 128 ? mixed3_fcorrect_kernel<NB, S, 128>
                                      : mixed3_fcorrect_kernel<NB, S, 256>)
                    : (block == 64    ? mixed3_correct_kernel<NB, S, 64>
                       : block == 128 ? mixed3_correct_kernel<NB, S, 128>
                                      : mixed3_correct_kernel<NB, S, 256>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<blocks, block, smem, s>>>(Q, (const float2*)Y, g.n[0], g.n[1], g.n[2], cp, gmax,
                                   ms.exps, ms.maxbits, (uint4*)ms.planes, ms.status);
  return cudaGetLastError();
}

cudaError_t launch_mixed3_correct(const Grid& g, int nb, int slices, double* Q, const void* Y,
                                  int gmax, const CorrParams& cp, MixedState& ms, int block,
                                  bool fused, cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  switch (nb * 16 + slices) {
#define RIDG_C3(NBV, SV) \
  case NBV * 16 + SV: return launch_correct3_t<NBV, SV>(g, Q, Y, gmax, cp, ms, block, fused, s);
    RIDG_C3(2, 2) RIDG_C3(2, 3) RIDG_C3(2, 4) RIDG_C3(2, 5) RIDG_C3(2, 6)
    RIDG_C3(3, 2) RIDG_C3(3, 3) RIDG_C3(3, 4) RIDG_C3(3, 5) RIDG_C3(3, 6)
#undef RIDG_C3
    default: return cudaErrorInvalidValue;
  }
}

template <int NB, int S>
static cudaError_t launch_refresh3_t(const Grid& g, const double* Q, MixedState& ms, cudaStream_t s) {
  constexpr int P = ((NB * NB * NB + 15) / 16) * 2;
  cudaError_t e = cudaMemsetAsync(ms.maxbits, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  state_max_kernel<<<256, 256, 0, s>>>(Q, g.ncell * NB * NB * NB, ms.maxbits);
  const unsigned blocks = (unsigned)((g.ncell * P + 127) / 128);
  state_digits3_kernel<NB, S><<<blocks, 128, 0, s>>>(Q, g.n[0], g.n[1], g.n[2], ms.maxbits, ms.exps,
                                                     (uint4*)ms.planes, ms.status);
  return cudaGetLastError();
}

cudaError_t launch_mixed3_refresh(const Grid& g, int nb, int slices, const double* Q,
                                  MixedState& ms, cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  switch (nb * 16 + slices) {
#define RIDG_R3(NBV, SV) \
  case NBV * 16 + SV: return launch_refresh3_t<NBV, SV>(g, Q, ms, s);
    RIDG_R3(2, 2) RIDG_R3(2, 3) RIDG_R3(2, 4) RIDG_R3(2, 5) RIDG_R3(2, 6)
    RIDG_R3(3, 2) RIDG_R3(3, 3) RIDG_R3(3, 4) RIDG_R3(3, 5) RIDG_R3(3, 6)
#undef RIDG_R3
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ridg
