// Mixed-precision RIDG step for a linear flux in 2D on the 5th-generation tensor cores
// (tcgen05 + TMA, sm_103a).
//
// What is computed.  Y[e][c] = sum_k G[c][k] X_e[k] for every cell e, where X_e holds the
// theta_S coefficients of the region cells upstream of e (Sec. 2.2, eq. region: the upwind
// box, 2 x 2 of the 3 x 3 vertex neighbours for a velocity with no zero component; the
// other cells' operator columns are exactly zero) and G is
// the centre-row region operator (the prediction of eq. pred_full_system for a linear
// flux), optionally composed with the linear correction functionals of Sec. 2.3 (volume
// term and upwind face traces) -- the "fused" step outputs [V | u_x | u_y].
//
// Split-operand refinement on BF16 tensor cores.  Every FP64 coefficient is written as a
// sum of S balanced base-256 digits, X = 2^s sum_a d_a 2^{-8(a+1)}, with one exponent s
// for the whole state (s = e + 1, 2^e > max |Q|): |d_0| <= 256, |d_a| <= 128.  The rows of
// G get their own exponents.  Digits are small integers, exact in BF16; digit products
// are exact; the K-sum of the products with equal weight a + c' = t is exact in the FP32
// accumulator for t <= 4 (bounded by (t+1) 144 2^16 < 2^24) and rounded far below the FP64
// target for t >= 5.  The diagonal sums acc_t live in TMEM (one block of columns per t);
// the epilogue recombines sum_t acc_t 2^{-8t} with error-free FP32 two-sums.
//
// Data path (one step = two kernels):
//   mixed_gemm_kernel      persistent, warp-specialised pipeline per CTA:
//     warp 0 / lane 0: TMA.  For every digit of an 8 x 16 cell tile the operand is one
//       3D TMA box of the ghost-padded digit planes [digit, 8-mode group][y + 2]
//       [(x + 2) x 8 modes], 8 x 18 cells, per x-offset of the box: they land in shared
//       memory exactly in the K-major core-matrix layout, so the A operand of the MMA for
//       region offset (ox, oy) is copy ox with its descriptor start moved by oy + 1 halo
//       rows (128 B, keeping every core matrix 128-byte aligned) -- an implicit im2col
//       without any copy by the SM.  Digits stream through a ring of slots, so the TMA runs a tile
//       ahead of the tensor core.
//     warp 1 / lane 0: MMA.  Descriptors are formed in registers (constant offsets).
//       S x (box cells) x (theta_pad / 16) tcgen05.mma (M = 128); B = operator digits stacked so the
//       pair (a, c') lands in TMEM block a + c'.  One commit per tile.
//     warps 2..9: epilogue (thread <-> TMEM lane <-> cell, two warps per lane quadrant);
//       TMEM is double-buffered.
//   mixed_correct_kernel   the correction from the fused outputs in double-float FP32 with
//       the final conservative state update in FP64, the new state's maximum, and the
//       digit planes of the new state for the next step's TMA.
// Every wait is bounded; on timeout a kernel raises a status bit, waits once more (bounded)
// for the tensor core, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "k_tc.cuh"
#include "ridg_internal.h"

namespace ridg {
namespace {


struct GemmLayout {
  int P, brows, slots, nmma, G, groups;
  uint32_t copy_bytes, slot_bytes, b_off, bbytes, bar_off, bytes;
};

// MMAs of digit a: nreg region offsets x k-steps x operator-digit chunks (N <= 256)
__host__ __device__ inline int gemm_nmma_digit(int S, int P, int nout_pad, int a, int nreg) {
  const int cmax = 256 / nout_pad;
  return nreg * (P / 2) * ((S - a + cmax - 1) / cmax);
}

// Shared memory: a ring of slots, each holding G digits of one tile (ncx x-shifted copies
// of the 8 x 18 halo box per digit, one per x-offset of the upwind box), then the operator
// digits of the box's nreg cells, then the barriers.  G is the largest group of digits for
// which two slots fit.
__host__ __device__ inline GemmLayout gemm_layout(int S, int thS, int nout_pad, int ncx, int nreg) {
  GemmLayout l;
  l.P = ((thS + 15) / 16) * 2;  // 8-mode groups after padding theta_S to a multiple of 16
  l.brows = S * nout_pad;
  l.nmma = 0;
  for (int a = 0; a < S; ++a) l.nmma += gemm_nmma_digit(S, l.P, nout_pad, a, nreg);
  l.bbytes = (uint32_t)nreg * l.P * l.brows * 16;
  const uint32_t digit_bytes = (uint32_t)ncx * l.P * kCopy * 16;  // one digit: ncx copies
  const uint32_t rest = l.bbytes + 256 + 1024;
  const uint32_t avail = rest < kSmemLimit ? kSmemLimit - rest : 0;
  int G = S;
  while (G > 1 && 2 * ((G * digit_bytes + 1023) & ~1023u) > avail) --G;
  l.G = G;
  l.groups = (S + G - 1) / G;
  l.copy_bytes = (uint32_t)G * l.P * kCopy * 16;      // G digits, one x-shifted copy
  l.slot_bytes = ((ncx * l.copy_bytes) + 1023) & ~1023u;
  int slots = (int)(avail / l.slot_bytes);
  l.slots = slots > kMaxSlots ? kMaxSlots : slots;
  l.b_off = (uint32_t)l.slots * l.slot_bytes;
  l.bar_off = (l.b_off + l.bbytes + 63) & ~63u;
  l.bytes = l.bar_off + 256;
  return l;
}

// ---------------------------------------------------------------------------------------
// the tensor-core contraction
// ---------------------------------------------------------------------------------------
// NREGC = 4: the 2 x 2 box of a velocity with no zero component, the offset loop unrolled
// (the single MMA-issuing thread is instruction-bound on a runtime loop: 27 vs 19 us per
// launch at 256^2, Q3); NREGC = 0: any box, runtime loop.
template <int NB, int NOUTP, bool OUTF2, int NREGC>
__global__ void __launch_bounds__(kGemmThreads, 1) mixed_gemm_kernel(
    const __grid_constant__ CUtensorMap dmap, const uint4* __restrict__ Bg,
    const double* __restrict__ rscale, const float* __restrict__ rowmul, int S, int nout,
    void* __restrict__ Yv, long long ystride_e, long long ystride_c, int* __restrict__ exps,
    unsigned long long* __restrict__ maxbits, int nx, int ny, RegionBox box, int* status) {
  constexpr int THS = NB * NB;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_base_sh;
  const int ox0 = box.lo[0], oy0 = box.lo[1];
  const int ncx = NREGC ? 2 : box.cnt[0], nreg = NREGC ? NREGC : box.n;
  const GemmLayout L = gemm_layout(S, THS, NOUTP, ncx, nreg);
  const int NSL = L.slots;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty;
  const int mytiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nitems = mytiles * L.groups;  // (tile, digit group) pairs of this CTA
  const int tcols = S * NOUTP;     // TMEM columns per stage
  const int tstages = 2 * tcols <= 512 ? 2 : 1;
  const int ncols = tstages * tcols <= 256 ? 256 : 512;
  // barriers: full[slot] (TMA landed), done[slot] (MMAs reading the slot complete),
  // tdone[2] (all MMAs of a tile complete), empty[2] (TMEM stage read out by the 256
  // epilogue threads), opload (operator digits + MMA table)
  const uint32_t bar = smem_u32(smem + L.bar_off);
  const uint32_t full0 = bar, done0 = bar + 8u * kMaxSlots, tdone0 = bar + 16u * kMaxSlots,
                 empty0 = tdone0 + 16u, opload = tdone0 + 32u;
  const uint32_t copy_bytes = L.copy_bytes;
  const int sexp = exps[0];  // exponent the digit planes were made with
  const bool f16 = exps[2] != 0;  // FP16 (else BF16) digit operands

  auto issue_item = [&](int item) {
    const int kk = item / L.groups, q = item % L.groups, sl = item % NSL;
    const int tile = blockIdx.x + kk * gridDim.x;
    const uint32_t dst = smem_u32(smem + sl * L.slot_bytes);
    const uint32_t fb = full0 + 8u * sl;
    mbar_expect_tx(fb, ncx * copy_bytes);  // out-of-range planes are zero-filled and counted
    const int x0 = (tile % ntx) * kTX, y0 = (tile / ntx) * kTY;
    // copy jx holds x-offset ox0 + jx: padded column x0 + 1 + ox0 + jx (x and the 8 modes
    // form one contiguous dimension, so the coordinate is a multiple of 8 elements)
    for (int jx = 0; jx < ncx; ++jx)
      tma_load_3d(dst + jx * copy_bytes, &dmap, (x0 + 1 + ox0 + jx) * 8, y0, q * L.G * L.P, fb);
  };

  if (tid == 0) {
    for (int i = 0; i < kMaxSlots; ++i) {
      mbar_init(full0 + 8u * i, 1);
      mbar_init(done0 + 8u * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tdone0 + 8u * i, 1);
      mbar_init(empty0 + 8u * i, 256);
    }
    mbar_init(opload, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // operator digits: one asynchronous bulk copy
    mbar_expect_tx(opload, L.bbytes);
    for (uint32_t off = 0; off < L.bbytes; off += 32768u)
      bulk_load(smem_u32(smem + L.b_off + off), (const unsigned char*)Bg + off,
                min(32768u, L.bbytes - off), opload);
    for (int i = 0; i < NSL && i < nitems; ++i) issue_item(i);
    // the later items' boxes: into L2 now, so that the ring's refills hit L2, not HBM
    for (int item = NSL; item < nitems; ++item) {
      const int kk = item / L.groups, q = item % L.groups;
      const int tile = blockIdx.x + kk * gridDim.x;
      const int x0 = (tile % ntx) * kTX, y0 = (tile / ntx) * kTY;
      for (int jx = 0; jx < ncx; ++jx)
        tma_prefetch_3d(&dmap, (x0 + 1 + ox0 + jx) * 8, y0, q * L.G * L.P);
    }
    if (OUTF2 && blockIdx.x == 0) {
      // rotate the running maximum: the correction that follows accumulates a fresh one
      maxbits[0] = maxbits[1];
      maxbits[1] = 0;
      exps[1] = sexp;  // exponent of this step's outputs, read by the correction
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: refill a slot once its MMAs are done ----------------
      bool ok = NSL >= 2;
      for (int item = NSL; item < nitems && ok; ++item) {
        const int p = item - NSL, sp = p % NSL;
        if (!mbar_wait_sleep(done0 + 8u * sp, (p / NSL) & 1)) { ok = false; break; }
        issue_item(item);
      }
      if (!ok) atomicOr(status, kStatusTimeout);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr int P = ((THS + 15) / 16) * 2;
      constexpr int KSTEPS = P / 2;
      constexpr int CMAX = 256 / NOUTP;
      const uint32_t brows = (uint32_t)L.brows;
      const uint64_t bdesc0 = smem_desc(smem_u32(smem + L.b_off), brows * 16, 128);
      bool ok = NSL >= 2 && mbar_wait(opload, 0);
      int item = 0;
      for (int k = 0; k < mytiles && ok; ++k) {
        const int ts = k % tstages;
        if (k >= tstages && !mbar_wait(empty0 + 8u * ts, ((k - tstages) / tstages) & 1)) {
          ok = false;
          break;
        }
        const uint32_t tst = tmem + (uint32_t)(ts * tcols);
        for (int q = 0; q < L.groups; ++q, ++item) {
          const int sl = item % NSL;
          if (!mbar_wait(full0 + 8u * sl, (item / NSL) & 1)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // A: LBO = plane stride inside a copy, SBO = one halo row of 8 cells (128 B)
          const uint64_t adesc0 = smem_desc(smem_u32(smem + sl * L.slot_bytes), kCopy * 16, 128);
          const uint32_t copy16 = copy_bytes / 16;
          const int a_end = min(S, (q + 1) * L.G);
          for (int a = q * L.G; a < a_end; ++a) {
            const uint32_t dig = (uint32_t)((a - q * L.G) * P * kCopy);
            for (int c0 = 0; c0 < S - a; c0 += CMAX) {
              const int nn = (min(S - a, c0 + CMAX) - c0) * NOUTP;
              const uint32_t idesc = idesc_digits(128, nn, f16);
              const uint32_t dcol = tst + (uint32_t)((a + c0) * NOUTP);
#pragma unroll
              for (int r = 0; r < (NREGC ? NREGC : nreg); ++r) {
                // box cell r: x-offset ox0 + r % ncx (copy r % ncx), y-offset oy0 + r / ncx
                // (descriptor start moved by oy0 + r / ncx + 1 halo rows)
                const int jx = r % ncx, ry = oy0 + r / ncx + 1;
#pragma unroll
                for (int j = 0; j < KSTEPS; ++j) {
                  const uint32_t aoff = (uint32_t)jx * copy16 + dig + (uint32_t)(2 * j * kCopy) +
                                        (uint32_t)(ry * kTX);
                  const uint32_t boff = (uint32_t)(r * P + 2 * j) * brows + (uint32_t)(c0 * NOUTP);
                  const uint32_t acc = (a == 0 && r == 0 && j == 0) ? 0u : 1u;
                  mma_bf16(dcol, adesc0 + aoff, bdesc0 + boff, idesc, acc);
                }
              }
            }
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  done0 + 8u * sl)
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
    // ---------------- epilogue: warps 2..9, two per TMEM lane quadrant ----------------
    const int quad = warp & 3;                 // lanes 32 quad .. this warp may read
    const int part = (warp - 2) >> 2;          // which half of the output columns
    const int cell = quad * 32 + lane;
    const int ix = cell % kTX, iy = cell / kTX;
    const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
      const int ts = k % tstages;
      if (!mbar_wait_sleep(tdone0 + 8u * ts, (k / tstages) & 1)) {
        if (lane == 0) atomicOr(status, kStatusTimeout);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tx = tile % ntx, ty = tile / ntx;
      const int gx = tx * kTX + ix, gy = ty * kTY + iy;
      const long long e = (long long)gy * nx + gx;
      const uint32_t tbase = lane_addr + (uint32_t)(ts * tcols);
#pragma unroll 1
      for (int cb = part * (NOUTP / 2); cb < (part + 1) * (NOUTP / 2); cb += 8) {
        if (cb >= nout) break;
        uint32_t raw[7][8];  // every diagonal block of these 8 columns, one wait
#pragma unroll
        for (int t = 0; t < 7; ++t)
          if (t < S) tmem_ld8_nowait(tbase + (uint32_t)(t * NOUTP + cb), raw[t]);
        tmem_wait_ld();
        float hi[8], lo[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          hi[c] = __uint_as_float(raw[0][c]);
          lo[c] = 0.f;
        }
        float w = 1.f;
#pragma unroll
        for (int t = 1; t < 7; ++t) {
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
          if (OUTF2) {
            // (hi, lo) scaled to the common row exponent; value = (hi + lo) 2^(s + gmax - 16)
            float2* y = (float2*)Yv + e * ystride_e + (long long)cb * ystride_c;
#pragma unroll
            for (int c = 0; c < 8; ++c)
              if (cb + c < nout) {
                const float m = rowmul[cb + c];
                y[c * ystride_c] = make_float2(hi[c] * m, lo[c] * m);
              }
          } else {
            double* y = (double*)Yv + e * ystride_e + (long long)cb * ystride_c;
            const double tscale = __longlong_as_double((long long)(sexp + 1023) << 52);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              if (cb + c < nout)
                y[c * ystride_c] = ((double)hi[c] + (double)lo[c]) * (tscale * rscale[cb + c]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(empty0 + 8u * ts);
    }
  }
  // drain: make sure no MMA is still writing TMEM before it is released (bounded)
  if (tid == 0 && mytiles > 0)
    mbar_wait(tdone0 + 8u * ((mytiles - 1) % tstages), ((mytiles - 1) / tstages) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------------------
// digit planes of the state (ghost-padded): plane (a * P + p), row (y + 1), column (x + 1)
// ---------------------------------------------------------------------------------------
template <int NB, int S>
__device__ __forceinline__ bool write_cell_digits(const double* q, int ix, int iy, int nx, int ny,
                                                  int s, uint4* __restrict__ planes, bool f16) {
  constexpr int THS = NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  const long long plane = (long long)(nx + 2) * (ny + 2);
  // padded positions holding this cell: itself and its periodic ghost copies
  int px[2] = {ix + 1, -1}, py[2] = {iy + 1, -1};
  if (ix == 0) px[1] = nx + 1;
  if (ix == nx - 1) px[1] = 0;
  if (iy == 0) py[1] = ny + 1;
  if (iy == ny - 1) py[1] = 0;
  bool fits = true;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = (p * 8 + j < THS) ? q[p * 8 + j] : 0.0;
    uint4 rows[S];
    fits &= make_digit_rows<S>(v, s, rows, f16);
#pragma unroll
    for (int a = 0; a < S; ++a) {
      uint4* base = planes + (long long)(a * P + p) * plane;
#pragma unroll
      for (int yi = 0; yi < 2; ++yi) {
        if (py[yi] < 0) continue;
#pragma unroll
        for (int xi = 0; xi < 2; ++xi) {
          if (px[xi] < 0) continue;
          base[(long long)py[yi] * (nx + 2) + px[xi]] = rows[a];
        }
      }
    }
  }
  return fits;
}

// digit rows of mode group p (8 coefficients v) of cell (ix, iy) and its ghost copies
template <int NB, int S>
__device__ __forceinline__ bool write_group_digits(const double* v, int p, int ix, int iy, int nx,
                                                   int ny, int s, uint4* __restrict__ planes,
                                                   bool f16) {
  constexpr int THS = NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  const long long plane = (long long)(nx + 2) * (ny + 2);
  int px[2] = {ix + 1, -1}, py[2] = {iy + 1, -1};
  if (ix == 0) px[1] = nx + 1;
  if (ix == nx - 1) px[1] = 0;
  if (iy == 0) py[1] = ny + 1;
  if (iy == ny - 1) py[1] = 0;
  uint4 rows[S];
  const bool fits = make_digit_rows<S>(v, s, rows, f16);
#pragma unroll
  for (int a = 0; a < S; ++a) {
    uint4* base = planes + (long long)(a * P + p) * plane;
#pragma unroll
    for (int yi = 0; yi < 2; ++yi) {
      if (py[yi] < 0) continue;
#pragma unroll
      for (int xi = 0; xi < 2; ++xi) {
        if (px[xi] < 0) continue;
        base[(long long)py[yi] * (nx + 2) + px[xi]] = rows[a];
      }
    }
  }
  return fits;
}

// digit planes of the current state from maxbits[1]; exps[0] = their exponent
template <int NB, int S>
__global__ void state_digits_kernel(const double* __restrict__ Q, int nx, int ny,
                                    const unsigned long long* maxbits, int* exps,
                                    uint4* __restrict__ planes, int* status) {
  constexpr int THS = NB * NB;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = exponent_above(maxbits[1]) + 1;
  if (e == 0) exps[0] = s;
  if (e >= (long long)nx * ny) return;
  double q[THS];
#pragma unroll
  for (int i = 0; i < THS; ++i) q[i] = Q[e * THS + i];
  const unsigned ue = (unsigned)e, uy = ue / (unsigned)nx;
  if (!write_cell_digits<NB, S>(q, (int)(ue - uy * (unsigned)nx), (int)uy, nx, ny, s, planes,
                                exps[2] != 0))
    atomicOr(status, kStatusRange);
}

// ---------------------------------------------------------------------------------------
// correction from the fused outputs.  Y holds, output-major, [V (theta_S) | u_x (NB) | u_y
// (NB)] per cell as double-float pairs (hi, lo) whose value is (hi + lo) 2^(s + gmax - 16)
// with s the exponent of this step's digit planes: V = sum_d nu_d (D along d) Wbar and u_d
// = nu_d trace(Wbar) on the upwind side of dim d (trace at +1 when a_d > 0, at -1 when
// a_d < 0).  The face value at i+1/2 in dim d is u_d of the upwind cell -- one stored pair
// per face, applied with opposite signs to both neighbours.  With phi_a(-1) = (-1)^a
// phi_a(+1) the update of mode (a, t) along d is phi_a(+1) (-F_{i+1/2} + (-1)^a F_{i-1/2}).
// The sums run in double-float FP32; the final state update is FP64.  The kernel then
// writes the new state's digit planes (exponent from the previous maximum plus one bit of
// headroom, checked) and accumulates the new maximum.
// ---------------------------------------------------------------------------------------
struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  float s2 = __fadd_rn(s, e);
  return DF{s2, __fsub_rn(e, __fsub_rn(s2, s))};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }

// (ch + cl) * (a.h + a.l) to double-float accuracy
__device__ __forceinline__ DF df_mul_const(float ch, float cl, DF a) {
  const float p = __fmul_rn(ch, a.h);
  float e = __fmaf_rn(ch, a.h, -p);
  e = __fmaf_rn(ch, a.l, e);
  e = __fmaf_rn(cl, a.h, e);
  const float s = __fadd_rn(p, e);
  return DF{s, __fsub_rn(e, __fsub_rn(s, p))};
}

// float * 2^k as a double, by exponent arithmetic on the bits (exact; 0 stays 0)
__device__ __forceinline__ double f2d_scaled(float f, int k) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e8 = (b >> 23) & 0xFF;
  if (e8 == 0) return 0.0;  // zero (denormal pairs do not occur: values are digit sums)
  const int e11 = (int)e8 - 127 + 1023 + k;
  if (e11 <= 0) return 0.0;
  const uint32_t hiw = (b & 0x80000000u) | ((uint32_t)e11 << 20) | ((b & 0x7FFFFFu) >> 3);
  const uint32_t low = (b & 0x7u) << 29;
  return __hiloint2double((int)hiw, (int)low);
}

// One thread per cell: dQ = V + the upwind face terms of both directions, summed in
// registers (every mode index a compile-time constant); the block's state rows are read and
// written coalesced through shared memory; then the cell's digit rows, group by group.
template <int NB, int S>
__global__ void __launch_bounds__(128) mixed_correct_kernel(
    double* __restrict__ Q, const float2* __restrict__ Y, int nx, int ny, CorrParams cp, int gmax,
    int sgnx, int sgny, int* __restrict__ exps, unsigned long long* __restrict__ maxbits,
    uint4* __restrict__ planes, int* status) {
  constexpr int THS = NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  constexpr int BT = 128;
  constexpr int PITCH = THS + 1;  // odd pitch: conflict-free row access
  __shared__ double sq[BT * PITCH];
  __shared__ unsigned long long shmax[4];
  const long long ncell = (long long)nx * ny;
  const long long e0 = (long long)blockIdx.x * BT;
  const int nblk = (int)min((long long)BT, ncell - e0);
  const int ys = exps[1];                                  // exponent of Y
  const int snext = exponent_above(maxbits[0]) + 1;        // exponent for the new digits
  // coalesced load of the block's state rows
  for (int i = threadIdx.x; i < nblk * THS; i += BT) sq[(i / THS) * PITCH + i % THS] = Q[e0 * THS + i];
  __syncthreads();
  const long long e = e0 + threadIdx.x;
  unsigned long long mymax = 0;
  bool fits = true;
  if (threadIdx.x < nblk) {
    const unsigned ue = (unsigned)e, uy = ue / (unsigned)nx;
    const int ix = (int)(ue - uy * (unsigned)nx), iy = (int)uy;
    DF dq[THS];
#pragma unroll
    for (int j = 0; j < THS; ++j) {
      const float2 y = Y[(long long)j * ncell + e];  // volume term V
      dq[j] = DF{y.x, y.y};
    }
#pragma unroll
    for (int dd = 0; dd < 2; ++dd) {
      const int sg = dd == 0 ? sgnx : sgny;
      if (sg == 0) continue;
      const int st = dd == 0 ? 1 : NB;
      int rx = ix, ry = iy, lx = ix, ly = iy;
      if (dd == 0) {
        if (sg > 0) lx = ix == 0 ? nx - 1 : ix - 1; else rx = ix + 1 == nx ? 0 : ix + 1;
      } else {
        if (sg > 0) ly = iy == 0 ? ny - 1 : iy - 1; else ry = iy + 1 == ny ? 0 : iy + 1;
      }
      const long long jr = (long long)ry * nx + rx, jl = (long long)ly * nx + lx;
      const float2* u = Y + (long long)(THS + dd * NB) * ncell;
      float2 fa[NB], fb[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        fa[t] = u[t * ncell + jr];
        fb[t] = u[t * ncell + jl];
      }
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const int base = dd == 0 ? t * NB : t;
        const DF fr = DF{fa[t].x, fa[t].y}, fl = DF{fb[t].x, fb[t].y};
        const DF w_even = df_add(fl, df_neg(fr));  // -F(i+1/2) + F(i-1/2)
        const DF w_odd = df_neg(df_add(fl, fr));   // -F(i+1/2) - F(i-1/2)
#pragma unroll
        for (int a2 = 0; a2 < NB; ++a2) {
          const DF w = (a2 & 1) ? w_odd : w_even;
          const DF c = (a2 == 0) ? w : df_mul_const(cp.eph[a2], cp.epl[a2], w);
          dq[base + a2 * st] = df_add(dq[base + a2 * st], c);
        }
      }
    }
    const int kfin = ys + gmax - 16;
    double* q = sq + threadIdx.x * PITCH;
#pragma unroll
    for (int pg = 0; pg < P; ++pg) {
      double qn[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int sm = pg * 8 + j;
        if (sm < THS) {
          double v = q[sm];
          v = v + f2d_scaled(dq[sm].h, kfin);
          v = v + f2d_scaled(dq[sm].l, kfin);
          q[sm] = v;
          qn[j] = v;
          const unsigned long long ab = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
          mymax = ab > mymax ? ab : mymax;
        } else {
          qn[j] = 0.0;
        }
      }
      fits &= write_group_digits<NB, S>(qn, pg, ix, iy, nx, ny, snext, planes, exps[2] != 0);
    }
  }
  if (!fits) atomicOr(status, kStatusRange);
  const unsigned long long bm = block_max_bits(mymax, shmax);
  if (threadIdx.x == 0) {
    atomicMax(maxbits + 1, bm);
    if (blockIdx.x == 0) exps[0] = snext;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nblk * THS; i += BT) Q[e0 * THS + i] = sq[(i / THS) * PITCH + i % THS];
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
bool mixed_supported(int dim, int nb, int nout) {
  if (dim == 3) return nb >= 2 && nb <= 3 && nout <= 64;
  return dim == 2 && nb >= 2 && nb <= 4 && nout <= 64;
}

static int nout_pad_of(int nout) { return nout <= 32 ? 32 : 64; }

int mixed_build(int dim, int nb, const std::vector<double>& G, int nout, int slices,
                const RegionBox& box, std::vector<unsigned short>& digits,
                std::vector<double>& rscale, std::vector<float>& rowmul, MixedOp& op, bool f16) {
  if (!mixed_supported(dim, nb, nout) || slices < 2 || slices > 7) return RIDG_EINVAL;
  if (dim == 3 && !mixed3_supported(nb, slices)) return RIDG_EINVAL;
  // region cells of G's columns: the upwind box, x fastest
  const int nreg = box.n, ncx = box.cnt[0];
  if (box.n < 1 || box.n > (dim == 3 ? 8 : 4) || (dim == 2 && box.cnt[2] != 1)) return RIDG_EINVAL;
  const int thS = dim == 3 ? nb * nb * nb : nb * nb, K = nreg * thS;
  if ((int)G.size() < nout * K) return RIDG_EINVAL;
  const int NOUTP = nout_pad_of(nout);
  // (3D: two TMEM stages of slices x NOUTP columns, and an MMA N of at most 256)
  if (slices * NOUTP > (dim == 3 ? 256 : 512)) return RIDG_EINVAL;
  const GemmLayout L = gemm_layout(slices, thS, NOUTP, ncx, nreg);
  const int tpad = L.P * 8;
  // digits in the shared-memory layout [region][k-chunk][row = c' * NOUTP + c][8]
  digits.assign((size_t)nreg * L.P * L.brows * 8, 0);
  rscale.assign(NOUTP, 0.0);
  rowmul.assign(NOUTP, 0.0f);
  std::vector<int> gexp(NOUTP, -100000);
  for (int c = 0; c < nout; ++c) {
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(G[(size_t)c * K + k]));
    int g = 0;
    if (mx > 0) std::frexp(mx, &g);  // mx < 2^g
    rscale[c] = std::ldexp(1.0, g - 2 * kBits);
    gexp[c] = mx > 0 ? g : -100000;
    for (int k = 0; k < K; ++k) {
      const int r = k / thS, s = k % thS;
      const int kp = r * tpad + s;  // padded column
      double v = std::ldexp(G[(size_t)c * K + k], -g);  // |v| < 1
      for (int cp = 0; cp < slices; ++cp) {
        double sc = std::ldexp(v, kBits);
        double d = (cp + 1 < slices) ? std::floor(sc + 0.5) : std::nearbyint(sc);
        v = sc - d;  // exact
        // |d| <= 256: exact in BF16 and in FP16
        unsigned short bits;
        if (f16) {
          const __half b = __float2half_rn((float)d);
          std::memcpy(&bits, &b, 2);
        } else {
          const __nv_bfloat16 b = __float2bfloat16_rn((float)d);
          std::memcpy(&bits, &b, 2);
        }
        const int row = cp * NOUTP + c;
        digits[((size_t)(kp / 8) * L.brows + row) * 8 + (kp % 8)] = bits;
      }
    }
  }
  if (dim == 2 && (L.bytes > kSmemLimit || L.slots < 2)) return RIDG_EINVAL;
  int gmax = -100000;
  for (int c = 0; c < nout; ++c) gmax = std::max(gmax, gexp[c]);
  if (gmax == -100000) gmax = 0;
  for (int c = 0; c < nout; ++c)
    rowmul[c] = gexp[c] == -100000 ? 0.0f
                                   : (gexp[c] - gmax < -126 ? 0.0f : std::ldexp(1.0f, gexp[c] - gmax));
  op.gmax = gmax;
  op.nout = nout;
  op.npad = NOUTP;
  op.K = K;
  op.Kpad = nreg * tpad;
  op.slices = slices;
  op.bits = kBits;
  return RIDG_OK;
}

size_t mixed_plane_bytes(const Grid& g, int nb, int slices) {
  const int thS = nb * nb, P = ((thS + 15) / 16) * 2;
  return (size_t)(g.n[0] + 2) * (g.n[1] + 2) * slices * P * 16;
}

int mixed_make_map(const Grid& g, int nb, int slices, int nout, void* planes, void* map_out) {
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
  const int thS = nb * nb, P = ((thS + 15) / 16) * 2;
  // dims (fastest first): padded x times 8 modes (BF16, contiguous), padded y, digit x
  // mode group; a box row is 8 cells x 8 modes = 128 B
  cuuint64_t dims[3] = {(cuuint64_t)(g.n[0] + 2) * 8, (cuuint64_t)(g.n[1] + 2),
                        (cuuint64_t)slices * P};
  cuuint64_t strides[2] = {(cuuint64_t)(g.n[0] + 2) * 16,
                           (cuuint64_t)(g.n[0] + 2) * (g.n[1] + 2) * 16};
  const GemmLayout L = gemm_layout(slices, thS, nout_pad_of(nout), g.box.cnt[0], g.box.n);
  cuuint32_t box[3] = {(cuuint32_t)kTX * 8, (cuuint32_t)kHY, (cuuint32_t)(L.G * P)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = ((EncodeFn)fn)((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes,
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RIDG_OK : RIDG_ECUDA;
}

template <int NB, int NOUTP, bool OUTF2>
static cudaError_t launch_gemm_t(const Grid& g, const void* map, const MixedOp& op, void* Y,
                                 long long ys_e, long long ys_c, MixedState& ms, cudaStream_t s) {
  const GemmLayout L = gemm_layout(op.slices, NB * NB, NOUTP, g.box.cnt[0], g.box.n);
  const bool box22 = g.box.cnt[0] == 2 && g.box.cnt[1] == 2;
  auto kern = box22 ? mixed_gemm_kernel<NB, NOUTP, OUTF2, 4> : mixed_gemm_kernel<NB, NOUTP, OUTF2, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = ((g.n[0] + kTX - 1) / kTX) * ((g.n[1] + kTY - 1) / kTY);
  const int grid = std::min(ntiles, sms);
  kern<<<grid, kGemmThreads, L.bytes, s>>>(*(const CUtensorMap*)map, (const uint4*)op.b_slices,
                                           op.row_scale, op.row_mul, op.slices, op.nout, Y, ys_e,
                                           ys_c, ms.exps, ms.maxbits, g.n[0], g.n[1], g.box,
                                           ms.status);
  return cudaGetLastError();
}

cudaError_t launch_mixed_gemm(const Grid& g, int nb, const MixedOp& op, MixedState& ms, void* Y,
                              long long ys_e, long long ys_c, bool fused, cudaStream_t s) {
  if (g.dim != 2 || g.box.n < 1 || g.box.n > 4 || op.K != g.box.n * nb * nb)
    return cudaErrorInvalidValue;
#define RIDG_GEMM_CASE(NBV, NP)                                                              \
  case NBV:                                                                                   \
    return fused ? launch_gemm_t<NBV, NP, true>(g, ms.map, op, Y, ys_e, ys_c, ms, s)          \
                 : launch_gemm_t<NBV, NP, false>(g, ms.map_pred, op, Y, ys_e, ys_c, ms, s);
  if (op.npad == 32) {
    switch (nb) { RIDG_GEMM_CASE(2, 32) RIDG_GEMM_CASE(3, 32) RIDG_GEMM_CASE(4, 32) }
  } else if (op.npad == 64) {
    switch (nb) { RIDG_GEMM_CASE(2, 64) RIDG_GEMM_CASE(3, 64) RIDG_GEMM_CASE(4, 64) RIDG_GEMM_CASE(5, 64) }
  }
#undef RIDG_GEMM_CASE
  return cudaErrorInvalidValue;
}

template <int NB, int S>
static cudaError_t launch_refresh_t(const Grid& g, const double* Q, MixedState& ms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ms.maxbits, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  state_max_kernel<<<256, 256, 0, s>>>(Q, g.ncell * NB * NB, ms.maxbits);
  const unsigned blocks = (unsigned)((g.ncell + 127) / 128);
  state_digits_kernel<NB, S><<<blocks, 128, 0, s>>>(Q, g.n[0], g.n[1], ms.maxbits, ms.exps,
                                                    (uint4*)ms.planes, ms.status);
  return cudaGetLastError();
}

template <int NB, int S>
static cudaError_t launch_correct_t(const Grid& g, double* Q, const void* Y, int gmax,
                                    const CorrParams& cp, int sgnx, int sgny, MixedState& ms,
                                    cudaStream_t s) {
  const unsigned blocks = (unsigned)((g.ncell + 127) / 128);  // one thread per cell
  mixed_correct_kernel<NB, S><<<blocks, 128, 0, s>>>(Q, (const float2*)Y, g.n[0], g.n[1], cp, gmax,
                                                     sgnx, sgny, ms.exps, ms.maxbits,
                                                     (uint4*)ms.planes, ms.status);
  return cudaGetLastError();
}

#define RIDG_NB_S_SWITCH(FN, ...)                                                             \
  switch (nb * 16 + slices) {                                                                 \
    case 2 * 16 + 2: return FN<2, 2>(__VA_ARGS__);                                            \
    case 2 * 16 + 3: return FN<2, 3>(__VA_ARGS__);                                            \
    case 2 * 16 + 4: return FN<2, 4>(__VA_ARGS__);                                            \
    case 2 * 16 + 5: return FN<2, 5>(__VA_ARGS__);                                            \
    case 2 * 16 + 6: return FN<2, 6>(__VA_ARGS__);                                            \
    case 2 * 16 + 7: return FN<2, 7>(__VA_ARGS__);                                            \
    case 3 * 16 + 2: return FN<3, 2>(__VA_ARGS__);                                            \
    case 3 * 16 + 3: return FN<3, 3>(__VA_ARGS__);                                            \
    case 3 * 16 + 4: return FN<3, 4>(__VA_ARGS__);                                            \
    case 3 * 16 + 5: return FN<3, 5>(__VA_ARGS__);                                            \
    case 3 * 16 + 6: return FN<3, 6>(__VA_ARGS__);                                            \
    case 3 * 16 + 7: return FN<3, 7>(__VA_ARGS__);                                            \
    case 4 * 16 + 2: return FN<4, 2>(__VA_ARGS__);                                            \
    case 4 * 16 + 3: return FN<4, 3>(__VA_ARGS__);                                            \
    case 4 * 16 + 4: return FN<4, 4>(__VA_ARGS__);                                            \
    case 4 * 16 + 5: return FN<4, 5>(__VA_ARGS__);                                            \
    case 4 * 16 + 6: return FN<4, 6>(__VA_ARGS__);                                            \
    case 4 * 16 + 7: return FN<4, 7>(__VA_ARGS__);                                            \
    case 5 * 16 + 2: return FN<5, 2>(__VA_ARGS__);                                            \
    case 5 * 16 + 3: return FN<5, 3>(__VA_ARGS__);                                            \
    case 5 * 16 + 4: return FN<5, 4>(__VA_ARGS__);                                            \
    case 5 * 16 + 5: return FN<5, 5>(__VA_ARGS__);                                            \
    case 5 * 16 + 6: return FN<5, 6>(__VA_ARGS__);                                            \
    case 5 * 16 + 7: return FN<5, 7>(__VA_ARGS__);                                            \
    default: break;                                                                           \
  }

cudaError_t launch_mixed_refresh(const Grid& g, int nb, int slices, const double* Q,
                                 MixedState& ms, cudaStream_t s) {
  if (g.dim != 2) return cudaErrorInvalidValue;
  RIDG_NB_S_SWITCH(launch_refresh_t, g, Q, ms, s)
  return cudaErrorInvalidValue;
}

cudaError_t launch_mixed_correct(const Grid& g, int nb, int slices, double* Q, const void* Y,
                                 int gmax, const CorrParams& cp, int sgnx, int sgny,
                                 MixedState& ms, cudaStream_t s) {
  if (g.dim != 2) return cudaErrorInvalidValue;
  RIDG_NB_S_SWITCH(launch_correct_t, g, Q, Y, gmax, cp, sgnx, sgny, ms, s)
  return cudaErrorInvalidValue;
}

}  // namespace ridg
