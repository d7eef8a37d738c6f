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
// by loading the plane z + oz.  The operator digits of all the box's offsets do not fit next
// to the state digits in shared memory, so they stream too:
//   A ring (4 slots): one digit of one input plane (one x-copy per x-offset of the box, each
//     8-mode groups x 8 x 18 cells: 18.4 KB at Q2 with two x-offsets), loaded by 4D TMA
//     boxes of the ghost-padded digit planes;
//   B stages (one per y-offset of the box): the operator digits of the x-offsets of one
//     (oz, oy) row (24.6 KB), one bulk copy each; stage oy is refilled for the next oz once
//     the last digit's MMAs on it are complete.
// The MMA issuer runs oz -> digit a -> oy -> ox -> k-step; the epilogue writes W-bar as
// double-float pairs with a common exponent, and mixed3_correct_kernel applies the correction
// in double-float FP32 (state update FP64) and writes the next step's digit planes.  Every
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

constexpr int kNA = 4;      // A slots
constexpr int kNBst = 3;    // B stages (one per y-offset)
constexpr int kNOUTP = 32;  // padded outputs (theta_S <= 27)

struct DF3 {
  float h, l;
};

struct Gemm3Layout {
  int P, brows;
  uint32_t copy_bytes, a_bytes, b_bytes, b_off, bar_off, bytes;
};

// ncx = x-offsets of the upwind box (x-shifted copies per A slot, operator blocks per B row)
__host__ __device__ inline Gemm3Layout gemm3_layout(int S, int thS, int ncx) {
  Gemm3Layout l;
  l.P = ((thS + 15) / 16) * 2;
  l.brows = S * kNOUTP;
  l.copy_bytes = (uint32_t)l.P * kCopy * 16;
  l.a_bytes = ((uint32_t)ncx * l.copy_bytes + 1023u) & ~1023u;
  l.b_bytes = (uint32_t)ncx * l.P * l.brows * 16;
  l.b_off = kNA * l.a_bytes;
  l.bar_off = (l.b_off + kNBst * l.b_bytes + 63u) & ~63u;
  l.bytes = l.bar_off + 256;
  return l;
}

// NCXC = 2: two x-offsets, the x loop unrolled; NCXC = 0: runtime count.
template <int NB, int NCXC>
__global__ void __launch_bounds__(kGemmThreads, 1) mixed3_gemm_kernel(
    const __grid_constant__ CUtensorMap dmap, const unsigned char* __restrict__ Bg,
    const float* __restrict__ rowmul, int S, int nout, float2* __restrict__ Y, int* __restrict__ exps,
    unsigned long long* __restrict__ maxbits, int nx, int ny, int nz, RegionBox box,
    int* status) {
  constexpr int THS = NB * NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  constexpr int KSTEPS = P / 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_base_sh;
  // the upwind box: offsets lo + 0 .. cnt - 1 per dimension (cnt 1 or 2, at most 3 B stages)
  const int ox0 = box.lo[0], oy0 = box.lo[1], oz0 = box.lo[2];
  const int ncx = NCXC ? NCXC : box.cnt[0], ncy = box.cnt[1], ncz = box.cnt[2];
  const Gemm3Layout L = gemm3_layout(S, THS, ncx);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty * nz;
  const int mytiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int tcols = S * kNOUTP;  // TMEM columns per stage (two stages)
  const uint32_t bar = smem_u32(smem + L.bar_off);
  const uint32_t afull0 = bar, afree0 = bar + 8u * kNA, bfull0 = bar + 16u * kNA,
                 bfree0 = bfull0 + 8u * kNBst, tdone0 = bfree0 + 8u * kNBst, tempty0 = tdone0 + 16u;
  const int sexp = exps[0];

  auto tile_origin = [&](int k, int& x0, int& y0, int& z0) {
    const int tile = blockIdx.x + k * gridDim.x;
    x0 = (tile % ntx) * kTX;
    y0 = ((tile / ntx) % nty) * kTY;
    z0 = tile / (ntx * nty);
  };

  if (tid == 0) {
    for (int i = 0; i < kNA; ++i) {
      mbar_init(afull0 + 8u * i, 1);
      mbar_init(afree0 + 8u * i, 1);
    }
    for (int i = 0; i < kNBst; ++i) {
      mbar_init(bfull0 + 8u * i, 1);
      mbar_init(bfree0 + 8u * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tdone0 + 8u * i, 1);
      mbar_init(tempty0 + 8u * i, 256);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (blockIdx.x == 0) {
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
      // ---------------- producer: B rows of offsets and A digit planes, in MMA order ----
      bool ok = true;
      int ia = 0;  // A items issued
      for (int k = 0; k < mytiles && ok; ++k) {
        int x0, y0, z0;
        tile_origin(k, x0, y0, z0);
        for (int jz = 0; jz < ncz && ok; ++jz) {
          const int use = k * ncz + jz;  // use count of every B stage
          for (int jy = 0; jy < ncy; ++jy) {
            if (use > 0 && !mbar_wait_sleep(bfree0 + 8u * jy, (use - 1) & 1)) { ok = false; break; }
            const uint32_t fb = bfull0 + 8u * jy;
            mbar_expect_tx(fb, L.b_bytes);
            const unsigned char* src = Bg + (size_t)(jz * ncy + jy) * L.b_bytes;
            const uint32_t dst = smem_u32(smem + L.b_off + jy * L.b_bytes);
            for (uint32_t off = 0; off < L.b_bytes; off += 32768u)
              bulk_load(dst + off, src + off, min(32768u, L.b_bytes - off), fb);
          }
          for (int a = 0; a < S && ok; ++a, ++ia) {
            const int sl = ia % kNA;
            if (ia >= kNA && !mbar_wait_sleep(afree0 + 8u * sl, ((ia / kNA) - 1) & 1)) { ok = false; break; }
            const uint32_t fa = afull0 + 8u * sl;
            mbar_expect_tx(fa, ncx * L.copy_bytes);  // out-of-range boxes are zero-filled and counted
            const uint32_t dst = smem_u32(smem + sl * L.a_bytes);
            // copy jx: x-offset ox0 + jx (padded column x0 + 1 + ox0 + jx, a multiple of 8
            // elements), plane z-offset oz0 + jz (padded plane z0 + 1 + oz0 + jz)
            for (int jx = 0; jx < ncx; ++jx)
              tma_load_4d(dst + jx * L.copy_bytes, &dmap, (x0 + 1 + ox0 + jx) * 8, y0,
                          z0 + 1 + oz0 + jz, a * P, fa);
          }
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
      int ia = 0;
      for (int k = 0; k < mytiles && ok; ++k) {
        const int ts = k & 1;
        if (k >= 2 && !mbar_wait(tempty0 + 8u * ts, ((k - 2) >> 1) & 1)) { ok = false; break; }
        const uint32_t tst = tmem + (uint32_t)(ts * tcols);
        for (int jz = 0; jz < ncz && ok; ++jz) {
          const int use = k * ncz + jz;
          for (int a = 0; a < S && ok; ++a, ++ia) {
            const int sl = ia % kNA;
            if (!mbar_wait(afull0 + 8u * sl, (ia / kNA) & 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // A: LBO = plane stride inside a copy, SBO = one halo row of 8 cells (128 B)
            const uint64_t adesc0 = smem_desc(smem_u32(smem + sl * L.a_bytes), kCopy * 16, 128);
            const uint32_t idesc = idesc_bf16(128, (S - a) * kNOUTP);
            const uint32_t dcol = tst + (uint32_t)(a * kNOUTP);
            for (int jy = 0; jy < ncy; ++jy) {
              if (a == 0) {
                if (!mbar_wait(bfull0 + 8u * jy, use & 1)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              }
              const uint64_t bdesc0 = smem_desc(smem_u32(smem + L.b_off + jy * L.b_bytes), brows * 16, 128);
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
              if (a == S - 1)
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        bfree0 + 8u * jy)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    afree0 + 8u * sl)
                : "memory");
          }
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
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;
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
      for (int cb = part * (kNOUTP / 2); cb < (part + 1) * (kNOUTP / 2); cb += 8) {
        if (cb >= nout) break;
        uint32_t raw[7][8];
#pragma unroll
        for (int t = 0; t < 7; ++t)
          if (t < S) tmem_ld8_nowait(tbase + (uint32_t)(t * kNOUTP + cb), raw[t]);
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
          // (hi, lo) scaled to the common row exponent; value = (hi + lo) 2^(s + gmax - 16)
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (cb + c < nout) {
              const float m = rowmul[cb + c];
              Y[(long long)(cb + c) * ncell + e] = make_float2(hi[c] * m, lo[c] * m);
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
__device__ __forceinline__ DF3 df3_mul(float ch, float cl, DF3 a) {
  const float p = __fmul_rn(ch, a.h);
  float e = __fmaf_rn(ch, a.h, -p);
  e = __fmaf_rn(ch, a.l, e);
  e = __fmaf_rn(cl, a.h, e);
  const float s = __fadd_rn(p, e);
  return DF3{s, __fsub_rn(e, __fsub_rn(s, p))};
}

__device__ __forceinline__ DF3 df3_add(DF3 a, DF3 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float s2 = __fadd_rn(s, e);
  return DF3{s2, __fsub_rn(e, __fsub_rn(s2, s))};
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

// Face values of the +d face of every cell for the NB^2 lines t crossing it:
// F[(d NT + t) cells + e] = nu_d^+ tr_+(W-bar_e)[t] + nu_d^- tr_-(W-bar_right)[t], one thread
// per (cell, d).  Each face value is computed once; both its cells read it.
template <int NB>
__global__ void __launch_bounds__(128) mixed3_faces_kernel(const float2* __restrict__ Y, int nx,
                                                           int ny, int nz, CorrParams cp,
                                                           float2* __restrict__ F) {
  constexpr int NT = NB * NB;
  const long long ncell = (long long)nx * ny * nz;
  const int dd = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const unsigned ue = (unsigned)e, ur = ue / (unsigned)nx;
  const int ix = (int)(ue - ur * (unsigned)nx), iy = (int)(ur % (unsigned)ny), iz = (int)(ur / (unsigned)ny);
  int rxi = ix, ryi = iy, rzi = iz;
  if (dd == 0) rxi = ix + 1 == nx ? 0 : ix + 1;
  if (dd == 1) ryi = iy + 1 == ny ? 0 : iy + 1;
  if (dd == 2) rzi = iz + 1 == nz ? 0 : iz + 1;
  const long long jr = ((long long)rzi * ny + ryi) * nx + rxi;
  const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
  const float nph = cp.nph[dd], npl = cp.npl[dd], nmh = cp.nmh[dd], nml = cp.nml[dd];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int base = t % st + (t / st) * st * NB;
    DF3 tp{0.f, 0.f}, tm{0.f, 0.f};
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const float sg = (b & 1) ? -1.f : 1.f;  // phi_b(-1) = (-1)^b phi_b(+1)
      const float2 yo = Y[(base + b * st) * ncell + e];
      const float2 yr = Y[(base + b * st) * ncell + jr];
      tp = df3_add(tp, df3_mul(cp.eph[b], cp.epl[b], DF3{yo.x, yo.y}));
      tm = df3_add(tm, df3_mul(sg * cp.eph[b], sg * cp.epl[b], DF3{yr.x, yr.y}));
    }
    const DF3 f = df3_add(df3_mul(nph, npl, tp), df3_mul(nmh, nml, tm));
    F[(long long)(dd * NT + t) * ncell + e] = make_float2(f.h, f.l);
  }
}

// The update: one thread per (cell, 8-mode group), the group uniform over a block and the P
// blocks of the same 128 cells adjacent in launch order (so that they share the cells' state
// rows in L2).  dQ = sum_d [(nu_d D[a][a-1]) W-bar(mode a-1 along d) + phi_a(+1) (s_a
// F(i - 1/2) - F(i + 1/2))], s_a = (-1)^a = phi_a(-1) / phi_a(+1), in double-float; Q += dQ
// in FP64; then the group's digit rows of the new state (and ghost copies) and the running
// maximum.  Degrees up to 2: a mode has at most one volume-term source per direction.
template <int NB, int S>
__global__ void __launch_bounds__(128) mixed3_correct_kernel(
    double* __restrict__ Q, const float2* __restrict__ Y, const float2* __restrict__ F, int nx,
    int ny, int nz, CorrParams cp, int gmax, int* __restrict__ exps,
    unsigned long long* __restrict__ maxbits, uint4* __restrict__ planes, int* status) {
  static_assert(NB <= 3, "one volume-term source per mode and direction");
  constexpr int THS = NB * NB * NB, NT = NB * NB;
  constexpr int P = ((THS + 15) / 16) * 2;
  __shared__ unsigned long long shmax[4];
  const long long ncell = (long long)nx * ny * nz;
  const int pg = (int)(blockIdx.x % P), m0 = 8 * pg;
  const long long e = (long long)(blockIdx.x / P) * blockDim.x + threadIdx.x;
  const int ys = exps[1];
  const int snext = exponent_above(maxbits[0]) + 1;
  unsigned long long mymax = 0;
  bool fits = true;
  if (e < ncell) {
    const unsigned ue = (unsigned)e, ur = ue / (unsigned)nx;
    const int ix = (int)(ue - ur * (unsigned)nx), iy = (int)(ur % (unsigned)ny), iz = (int)(ur / (unsigned)ny);
    // left neighbours along x, y, z (periodic)
    long long jl[3];
    jl[0] = ix == 0 ? e + (nx - 1) : e - 1;
    jl[1] = iy == 0 ? e + (long long)(ny - 1) * nx : e - nx;
    jl[2] = iz == 0 ? e + (long long)(nz - 1) * nx * ny : e - (long long)nx * ny;
    DF3 dq[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) dq[j] = DF3{0.f, 0.f};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const int st = dd == 0 ? 1 : (dd == 1 ? NB : NB * NB);
      const float2* Fd = F + (long long)dd * NT * ncell;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int sm = m0 + j;
        if (sm >= THS) continue;
        const int a = (sm / st) % NB;                          // index along d
        const int base = sm - a * st;                          // the line's first mode
        const int t = (base % st) + (base / (st * NB)) * st;   // line index
        DF3 v = dq[j];
        if (a >= 1) {
          const float2 y = Y[(base + (a - 1) * st) * ncell + e];
          v = df3_add(v, df3_mul(cp.vdh[dd][a], cp.vdl[dd][a], DF3{y.x, y.y}));
        }
        const float2 fp = Fd[t * ncell + e];
        const float2 fm = Fd[t * ncell + jl[dd]];
        const float sg = (a & 1) ? -1.f : 1.f;
        const DF3 df = df3_add(DF3{sg * fm.x, sg * fm.y}, DF3{-fp.x, -fp.y});
        dq[j] = df3_add(v, df3_mul(cp.eph[a], cp.epl[a], df));
      }
    }
    const int kfin = ys + gmax - 16;
    double qn[8];
    double* q = Q + e * THS;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (m0 + j < THS) {
        double v = q[m0 + j];
        v = v + f2d_scale(dq[j].h, kfin);
        v = v + f2d_scale(dq[j].l, kfin);
        q[m0 + j] = v;
        qn[j] = v;
        const unsigned long long ab = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
        mymax = ab > mymax ? ab : mymax;
      } else {
        qn[j] = 0.0;
      }
    }
    uint4 rows[S];
    fits = make_digit_rows<S>(qn, snext, rows);
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
  if (!make_digit_rows<S>(v, s, rows)) atomicOr(status, kStatusRange);
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

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
bool mixed3_supported(int nb, int slices) {
  if (nb < 2 || nb > 3 || slices < 2 || slices > 6) return false;
  return gemm3_layout(slices, nb * nb * nb, 3).bytes <= kSmemLimit;  // widest box
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
                                  cudaStream_t s) {
  const Gemm3Layout L = gemm3_layout(op.slices, NB * NB * NB, g.box.cnt[0]);
  // one CTA per SM: each allocates all 512 TMEM columns, so a second CTA on the SM would
  // only wait for them -- ask for more than half the shared memory
  const uint32_t smem = std::max<uint32_t>(L.bytes, 117u * 1024u);
  auto kern = g.box.cnt[0] == 2 ? mixed3_gemm_kernel<NB, 2> : mixed3_gemm_kernel<NB, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = ((g.n[0] + kTX - 1) / kTX) * ((g.n[1] + kTY - 1) / kTY) * g.n[2];
  const int grid = std::min(ntiles, sms);
  kern<<<grid, kGemmThreads, smem, s>>>(*(const CUtensorMap*)ms.map,
                                        (const unsigned char*)op.b_slices, op.row_mul, op.slices,
                                        op.nout, (float2*)Y, ms.exps, ms.maxbits, g.n[0], g.n[1],
                                        g.n[2], g.box, ms.status);
  return cudaGetLastError();
}

cudaError_t launch_mixed3_gemm(const Grid& g, int nb, const MixedOp& op, MixedState& ms, void* Y,
                               cudaStream_t s) {
  if (g.dim != 3 || g.box.n < 1 || g.box.n > 8 || op.K != g.box.n * nb * nb * nb)
    return cudaErrorInvalidValue;
  switch (nb) {
    case 2: return launch_gemm3_t<2>(g, op, ms, Y, s);
    case 3: return launch_gemm3_t<3>(g, op, ms, Y, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NB, int S>
static cudaError_t launch_correct3_t(const Grid& g, double* Q, const void* Y, void* F, int gmax,
                                     const CorrParams& cp, MixedState& ms, cudaStream_t s) {
  constexpr int P = ((NB * NB * NB + 15) / 16) * 2;
  const dim3 fblocks((unsigned)((g.ncell + 127) / 128), 3);
  mixed3_faces_kernel<NB><<<fblocks, 128, 0, s>>>((const float2*)Y, g.n[0], g.n[1], g.n[2], cp,
                                                  (float2*)F);
  const unsigned blocks = (unsigned)((g.ncell + 127) / 128) * P;
  mixed3_correct_kernel<NB, S><<<blocks, 128, 0, s>>>(Q, (const float2*)Y, (const float2*)F,
                                                      g.n[0], g.n[1], g.n[2], cp, gmax, ms.exps,
                                                      ms.maxbits, (uint4*)ms.planes, ms.status);
  return cudaGetLastError();
}

cudaError_t launch_mixed3_correct(const Grid& g, int nb, int slices, double* Q, const void* Y,
                                  void* F, int gmax, const CorrParams& cp, MixedState& ms,
                                  cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  switch (nb * 16 + slices) {
#define RIDG_C3(NBV, SV) \
  case NBV * 16 + SV: return launch_correct3_t<NBV, SV>(g, Q, Y, F, gmax, cp, ms, s);
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
