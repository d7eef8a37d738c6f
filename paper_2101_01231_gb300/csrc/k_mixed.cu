// Mixed-precision linear prediction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// What is computed.  Y[e][c] = sum_k G[c][k] X_e[k] for every cell e of a 2D mesh, where X_e
// holds the theta_S coefficients of the 3 x 3 vertex neighbours of e (Sec. 2.2, eq. region)
// and G is any operator with K = 9 theta_S columns -- the centre rows of the region
// solution operator (the prediction of eq. pred_full_system for a linear flux), or those
// rows composed with the linear correction functionals (volume term and upwind face
// traces of Sec. 2.3), which is what the fused step uses.
//
// How (split-operand refinement on BF16 tensor cores).  Each FP64 operand is written as a
// short sum of 8-bit "digits" times powers of two: for a tile of cells, X = 2^s sum_a
// d_a 2^{-8(a+1)} with s the tile's largest exponent, |d_0| <= 256, |d_a| <= 128 (balanced,
// rounded), and likewise each row of G with its own exponent.  Digits are small integers,
// exact in BF16, so every digit product is exact and the K-sum of products with equal
// digit weight a + c' = t is exact in the FP32 accumulator for t <= 4 (bounded by
// (t+1) 144 2^16 < 2^24) and rounded far below the FP64 target for t >= 5.  The diagonal
// sums acc_t live in TMEM (one block of columns per t); the epilogue recombines
// sum_t acc_t 2^{-8t} with error-free FP32 two-sums and scales by 2^{s + g_c - 16} in FP64.
//
// Data path per CTA (persistent over 8 x 16 cell tiles, 128 threads = 128 TMEM lanes):
//   1. the tile's 10 x 18 halo of FP64 coefficients is read from HBM (periodic wrap);
//   2. the halo is converted once to fixed point and split into S digit planes laid out
//      [digit][mode-group of 8][halo cell][8 modes] in shared memory;
//   3. the A operand of every MMA is read straight from the digit planes: region offset
//      (ox, oy) is a shift of the descriptor start address, the 8-row core matrices are 8
//      consecutive halo cells (16 B apart) and the 8-row groups are halo rows (160 B apart)
//      -- an implicit im2col, no copy;
//   4. one thread issues S x 9 x (theta_pad / 16) tcgen05.mma (M = 128) with B = the
//      operator digits stacked [G-digit 0 .. S-1-a] so digit pair (a, c') lands in TMEM
//      block a + c'; a single commit signals the mbarrier;
//   5. the epilogue reads TMEM with tcgen05.ld (thread t <-> cell t), recombines and writes
//      Y in FP64.
// Every wait on the mbarrier is bounded; on timeout the kernel raises a status flag, waits
// (bounded) once more for the tensor core, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ridg_internal.h"

namespace ridg {
namespace {

constexpr int kTX = 8, kTY = 16;                 // cells per tile in x, y (128 = MMA M)
constexpr int kHX = kTX + 2, kHY = kTY + 2;      // halo
constexpr int kHalo = kHX * kHY;                 // 180 halo cells
constexpr int kThreads = 256;                    // 8 warps: 2 per TMEM lane quadrant
constexpr int kBits = 8;                         // digit width
constexpr long kWaitLimit = 1L << 22;            // bounded mbarrier polls (well under a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // SWIZZLE_NONE, K-major: LBO = byte stride between core matrices along K,
  // SBO = byte stride between 8-row groups along M/N; bits 46-47 = descriptor version 1.
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  // kind::f16: D = F32 (bit 4), A = B = BF16 (bits 7, 10), both K-major, N >> 3 at bit 17,
  // M >> 4 at bit 24
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// error-free sum of two floats (Knuth): a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FP64 -> fixed point with L fraction bits relative to 2^s (round half up), from the bits
__device__ __forceinline__ long long to_fixed(double x, int s, int L) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero / subnormal: far below the tile's scale
  const long long mant = (long long)((u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = ex - 1075 + L - s;
  long long F;
  if (sh >= 0) {
    F = mant << sh;
  } else if (sh > -63) {
    F = (mant + (1LL << (-sh - 1))) >> (-sh);
  } else {
    F = 0;
  }
  return (u >> 63) ? -F : F;
}

struct MixedLayout {
  int S, P, nout_pad, brows;
  uint32_t digits_off, b_off, bytes;
};

__host__ __device__ inline MixedLayout mixed_layout(int S, int thS, int nout_pad) {
  MixedLayout l;
  l.S = S;
  l.P = ((thS + 15) / 16) * 2;  // 8-mode groups after padding theta_S to a multiple of 16
  l.nout_pad = nout_pad;
  l.brows = S * nout_pad;
  l.digits_off = 0;
  const uint32_t digits = (uint32_t)S * l.P * kHalo * 16;
  l.b_off = (digits + 1023) & ~1023u;
  const uint32_t bbytes = (uint32_t)9 * l.P * l.brows * 16;
  l.bytes = l.b_off + bbytes;
  return l;
}

// one work item = 8 consecutive modes (one core-matrix row) of one halo cell
constexpr int kMaxItems = 3;  // ceil(180 * P / 256) for P <= 4

template <int NB, int NOUTP, bool OUTF2>
__global__ void __launch_bounds__(kThreads, 2) predict_mixed_kernel(
    const double* __restrict__ Q, const uint4* __restrict__ Bg, const double* __restrict__ rscale,
    const float* __restrict__ rowmul, int S, int nout, void* __restrict__ Yv, long long ystride_e,
    long long ystride_c, int* __restrict__ texp, int nx, int ny, int* status) {
  constexpr int THS = NB * NB;
  constexpr int TPAD = ((THS + 15) / 16) * 16;
  constexpr int P = TPAD / 8;
  constexpr int KSTEPS = TPAD / 16;
  constexpr int NITEMS = kHalo * P;
  constexpr int IPT = (NITEMS + kThreads - 1) / kThreads;  // items per thread
  static_assert(IPT <= kMaxItems, "too many halo items per thread");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ unsigned long long red[kThreads / 32];
  const MixedLayout L = mixed_layout(S, THS, NOUTP);
  unsigned char* digits = smem + L.digits_off;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty;
  const int ncols = NOUTP * 8 > 256 ? 512 : 256;  // TMEM columns: >= S * NOUTP (S <= 7)

  // operator digits -> shared memory (once per CTA)
  {
    uint4* bs = (uint4*)(smem + L.b_off);
    const int nb16 = 9 * P * L.brows;
    for (int i = tid; i < nb16; i += kThreads) bs[i] = Bg[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const int Lfix = kBits * S;
  bool ok = true;
  uint32_t phase = 0;

  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int tx = tile % ntx, ty = tile / ntx;
    // 1. halo values of this thread's items (8 modes of one halo cell each), and the max
    double v[IPT][8];
    unsigned long long mx = 0;
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int item = tid + it * kThreads;
      const int h = item % kHalo, p = item / kHalo;
      int gx = tx * kTX - 1 + h % kHX, gy = ty * kTY - 1 + h / kHX;
      while (gx < 0) gx += nx;
      while (gx >= nx) gx -= nx;
      while (gy < 0) gy += ny;
      while (gy >= ny) gy -= ny;
      const double* q = Q + ((long long)gy * nx + gx) * THS + p * 8;
      if (item < NITEMS) {
        if (THS % 8 == 0) {
          const double2* q2 = (const double2*)q;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            double2 t = __ldg(q2 + j);
            v[it][2 * j] = t.x;
            v[it][2 * j + 1] = t.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) v[it][j] = (p * 8 + j < THS) ? __ldg(q + j) : 0.0;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[it][j] = 0.0;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const unsigned long long a =
            (unsigned long long)__double_as_longlong(v[it][j]) & 0x7FFFFFFFFFFFFFFFULL;
        mx = a > mx ? a : mx;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < kThreads / 32; ++w) mx = red[w] > mx ? red[w] : mx;
    // tile exponent: max|X| < 2^s
    const int sexp = mx == 0 ? 0 : (int)((mx >> 52) & 0x7FF) - 1022;
    // 2. fixed point (L = 8 S fraction bits), balanced base-256 digits from its bytes, and
    //    the digit planes [digit][mode group][halo cell][8 modes] (one 16 B store each)
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int item = tid + it * kThreads;
      uint32_t packed[7][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long F = to_fixed(v[it][j], sexp, Lfix);
        const uint32_t lo32 = (uint32_t)F, hi32 = (uint32_t)((unsigned long long)F >> 32);
        const int neg = (int)(hi32 >> 31);
        int carry = 0;
        int d[7];
#pragma unroll
        for (int a = 6; a >= 0; --a) {
          if (a < S) {
            const int k = S - 1 - a;  // byte index of digit a
            const uint32_t byte = (k < 4 ? (lo32 >> (8 * k)) : (hi32 >> (8 * (k - 4)))) & 0xFFu;
            if (a > 0) {
              const int t = (int)byte + carry;
              carry = (t + 128) >> 8;
              d[a] = t - (carry << 8);
            } else {
              d[0] = (int)byte - (neg << 8) + carry;
            }
          } else {
            d[a] = 0;
          }
        }
#pragma unroll
        for (int a = 0; a < 7; ++a) {
          // |d| <= 256: exact in FP32 by the 1.5 * 2^23 trick, and its BF16 is the top half
          const uint32_t b = __float_as_uint(__int_as_float(0x4B400000 + d[a]) - 12582912.0f) >> 16;
          if (j & 1)
            packed[a][j / 2] |= b << 16;
          else
            packed[a][j / 2] = b;
        }
      }
      if (item < NITEMS) {
        const int h = item % kHalo, p = item / kHalo;
#pragma unroll
        for (int a = 0; a < 7; ++a)
          if (a < S) {
            uint4* dst = (uint4*)(digits + ((size_t)(a * P + p) * kHalo + h) * 16);
            *dst = make_uint4(packed[a][0], packed[a][1], packed[a][2], packed[a][3]);
          }
      }
    }
    if (OUTF2 && tid == 0) texp[tile] = sexp;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 3./4. MMAs, issued by one thread
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dbase = smem_u32(digits), bbase = smem_u32(smem + L.b_off);
      const uint32_t a_lbo = kHalo * 16, a_sbo = kHX * 16;
      const uint32_t b_lbo = (uint32_t)L.brows * 16, b_sbo = 128;
      constexpr int CMAX = 256 / NOUTP;
      for (int a = 0; a < S; ++a) {
        for (int r = 0; r < 9; ++r) {
          const int ox = r % 3, oy = r / 3;  // halo shift (offset + 1)
          for (int j = 0; j < KSTEPS; ++j) {
            const uint32_t a_addr = dbase + (uint32_t)(((a * P + 2 * j) * kHalo + oy * kHX + ox) * 16);
            const uint64_t ad = smem_desc(a_addr, a_lbo, a_sbo);
            const int kc = r * P + 2 * j;  // k-chunk of the operator
            for (int c0 = 0; c0 < S - a; c0 += CMAX) {
              const int c1 = min(S - a, c0 + CMAX);
              const int n = (c1 - c0) * NOUTP;
              const uint32_t b_addr = bbase + (uint32_t)(kc * L.brows + c0 * NOUTP) * 16;
              const uint64_t bd = smem_desc(b_addr, b_lbo, b_sbo);
              const uint32_t acc = (a == 0 && r == 0 && j == 0) ? 0u : 1u;
              mma_bf16(tmem + (uint32_t)((a + c0) * NOUTP), ad, bd, idesc_bf16(128, n), acc);
            }
          }
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar))
          : "memory");
    }
    // 5. epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 cells) and half of the
    //    columns of every block
    if (!mbar_wait(smem_u32(&mbar), phase)) {
      ok = false;
      if (tid == 0) atomicOr(status, 2);
      mbar_wait(smem_u32(&mbar), phase);  // one more bounded wait before releasing TMEM
      break;
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
      const int quad = warp & 3, half = warp >> 2;
      const int cell = quad * 32 + lane;
      const int ix = cell % kTX, iy = cell / kTX;
      const int gx = tx * kTX + ix, gy = ty * kTY + iy;
      const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
      const long long e = (long long)gy * nx + gx;
#pragma unroll 1
      for (int cb = half * (NOUTP / 2); cb < (half + 1) * (NOUTP / 2); cb += 16) {
        float hi[16], lo[16], vv[16];
        tmem_ld16(lane_addr + (uint32_t)cb, hi);
#pragma unroll
        for (int c = 0; c < 16; ++c) lo[c] = 0.f;
        float w = 1.f;
        for (int t = 1; t < S; ++t) {
          w *= 1.f / 256.f;
          tmem_ld16(lane_addr + (uint32_t)(t * NOUTP + cb), vv);
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            float s2, e2;
            two_sum(hi[c], vv[c] * w, s2, e2);
            hi[c] = s2;
            lo[c] += e2;
          }
        }
        if (gx < nx && gy < ny) {
          if (OUTF2) {
            // (hi, lo) scaled to the common row exponent; value = (hi + lo) 2^(s + gmax - 16)
            float2* y = (float2*)Yv + e * ystride_e + (long long)cb * ystride_c;
#pragma unroll
            for (int c = 0; c < 16; ++c)
              if (cb + c < nout) {
                const float m = rowmul[cb + c];
                y[c * ystride_c] = make_float2(hi[c] * m, lo[c] * m);
              }
          } else {
            double* y = (double*)Yv + e * ystride_e + (long long)cb * ystride_c;
            const double tscale = __longlong_as_double((long long)(sexp + 1023) << 52);
#pragma unroll
            for (int c = 0; c < 16; ++c)
              if (cb + c < nout)
                y[c * ystride_c] = ((double)hi[c] + (double)lo[c]) * (tscale * rscale[cb + c]);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------------------
// correction from the fused outputs.  Y holds, output-major, [V (theta_S) | u_x (NB) | u_y
// (NB)] per cell as double-float pairs (hi, lo) whose value is (hi + lo) 2^(texp + gmax - 16)
// with texp the exponent of the cell's tile: V = sum_d nu_d (D along d) Wbar, and u_d =
// nu_d trace(Wbar) on the upwind side of dim d (trace at +1 when a_d > 0, at -1 when
// a_d < 0).  The face value at i+1/2 in dim d is u_d of the upwind cell -- one stored pair
// per face, applied with opposite signs to both neighbours.  With phi_a(-1) = (-1)^a
// phi_a(+1) the update of mode (a, t) along d is phi_a(+1) (-F_{i+1/2} + (-1)^a F_{i-1/2}).
// The sums run in double-float FP32 after aligning every pair to the largest exponent
// involved (power-of-two scaling, exact); only the final state update is FP64.
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

__device__ __forceinline__ DF df_scale(DF a, float m) { return DF{a.h * m, a.l * m}; }

// exact power of two 2^k as a float for k in [-126, 127]; 0 below
__device__ __forceinline__ float pow2f(int k) {
  return k < -126 ? 0.f : __uint_as_float((uint32_t)(k + 127) << 23);
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

template <int NB>
__global__ void __launch_bounds__(128) correct_fused_kernel(double* __restrict__ Q,
                                                            const float2* __restrict__ Y,
                                                            const int* __restrict__ texp,
                                                            int nx, int ny, CorrParams cp,
                                                            int gmax, int sgnx, int sgny) {
  constexpr int THS = NB * NB;
  constexpr int PITCH = THS + 1;  // odd pitch: conflict-free row access
  __shared__ double sq[128 * PITCH];
  const long long ncell = (long long)nx * ny;
  const long long e0 = (long long)blockIdx.x * 128;
  const int nblk = (int)min((long long)128, ncell - e0);
  const int ntx = (nx + kTX - 1) / kTX;
  // coalesced load of the block's state rows
  for (int i = threadIdx.x; i < nblk * THS; i += 128) sq[(i / THS) * PITCH + i % THS] = Q[e0 * THS + i];
  __syncthreads();
  const long long e = e0 + threadIdx.x;
  if (threadIdx.x < nblk) {
    const int ix = (int)(e % nx), iy = (int)(e / nx);
    // the cells whose stored values enter: own, and per dim the upwind cells of both faces
    long long jr[2], jl[2];
    int kr[2], kl[2];
    const int kown = texp[(ix / kTX) + (iy / kTY) * ntx];
    int kmax = kown;
#pragma unroll
    for (int dd = 0; dd < 2; ++dd) {
      const int sg = dd == 0 ? sgnx : sgny;
      int rx = ix, ry = iy, lx = ix, ly = iy;
      if (dd == 0) {
        if (sg > 0) lx = ix == 0 ? nx - 1 : ix - 1; else rx = ix + 1 == nx ? 0 : ix + 1;
      } else {
        if (sg > 0) ly = iy == 0 ? ny - 1 : iy - 1; else ry = iy + 1 == ny ? 0 : iy + 1;
      }
      jr[dd] = (long long)ry * nx + rx;
      jl[dd] = (long long)ly * nx + lx;
      kr[dd] = texp[(rx / kTX) + (ry / kTY) * ntx];
      kl[dd] = texp[(lx / kTX) + (ly / kTY) * ntx];
      if (sg != 0) kmax = max(kmax, max(kr[dd], kl[dd]));
    }
    DF dq[THS];
    const float mown = pow2f(kown - kmax);
#pragma unroll
    for (int s = 0; s < THS; ++s) {
      const float2 y = Y[s * ncell + e];  // volume term V
      dq[s] = df_scale(DF{y.x, y.y}, mown);
    }
#pragma unroll
    for (int dd = 0; dd < 2; ++dd) {
      const int sg = dd == 0 ? sgnx : sgny;
      if (sg == 0) continue;
      const int st = dd == 0 ? 1 : NB;
      const float mr = pow2f(kr[dd] - kmax), ml = pow2f(kl[dd] - kmax);
      const float2* u = Y + (long long)(THS + dd * NB) * ncell;
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const float2 a = u[t * ncell + jr[dd]], b = u[t * ncell + jl[dd]];
        const DF fr = df_scale(DF{a.x, a.y}, mr), fl = df_scale(DF{b.x, b.y}, ml);
        const DF w_even = df_add(fl, df_neg(fr));          // -F(i+1/2) + F(i-1/2)
        const DF w_odd = df_neg(df_add(fl, fr));           // -F(i+1/2) - F(i-1/2)
        const int base = dd == 0 ? t * NB : t;
#pragma unroll
        for (int a2 = 0; a2 < NB; ++a2) {
          const DF w = (a2 & 1) ? w_odd : w_even;
          const DF c = (a2 == 0) ? w : df_mul_const(cp.eph[a2], cp.epl[a2], w);
          dq[base + a2 * st] = df_add(dq[base + a2 * st], c);
        }
      }
    }
    const int kfin = kmax + gmax - 16;
    double* q = sq + threadIdx.x * PITCH;
#pragma unroll
    for (int s = 0; s < THS; ++s) {
      double v = q[s];
      v = v + f2d_scaled(dq[s].h, kfin);
      v = v + f2d_scaled(dq[s].l, kfin);
      q[s] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nblk * THS; i += 128) Q[e0 * THS + i] = sq[(i / THS) * PITCH + i % THS];
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
bool mixed_supported(int dim, int nb, int nout) {
  return dim == 2 && nb >= 2 && nb <= 5 && nout <= 64;
}

static int nout_pad_of(int nout) { return nout <= 32 ? 32 : 64; }

int mixed_build(int dim, int nb, const std::vector<double>& G, int nout, int slices,
                std::vector<unsigned short>& digits, std::vector<double>& rscale,
                std::vector<float>& rowmul, MixedOp& op) {
  if (!mixed_supported(dim, nb, nout) || slices < 2 || slices > 7) return RIDG_EINVAL;
  const int thS = nb * nb, K = 9 * thS;
  if ((int)G.size() < nout * K) return RIDG_EINVAL;
  const int NOUTP = nout_pad_of(nout);
  if (slices * NOUTP > 512) return RIDG_EINVAL;
  const MixedLayout L = mixed_layout(slices, thS, NOUTP);
  const int tpad = L.P * 8;
  // digits in the shared-memory layout [k-chunk][row = c' * NOUTP + c][8]
  digits.assign((size_t)9 * L.P * L.brows * 8, 0);
  rscale.assign(NOUTP, 0.0);
  rowmul.assign(NOUTP, 0.0f);
  std::vector<int> gexp(NOUTP, -100000);
  for (int c = 0; c < nout; ++c) {
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(G[(size_t)c * K + k]));
    int g = 0;
    if (mx > 0) {
      std::frexp(mx, &g);  // mx < 2^g
    }
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
        __nv_bfloat16 b = __float2bfloat16_rn((float)d);
        unsigned short bits;
        std::memcpy(&bits, &b, 2);
        const int row = cp * NOUTP + c;
        digits[((size_t)(kp / 8) * L.brows + row) * 8 + (kp % 8)] = bits;
      }
    }
  }
  int gmax = -100000;
  for (int c = 0; c < nout; ++c) gmax = std::max(gmax, gexp[c]);
  if (gmax == -100000) gmax = 0;
  for (int c = 0; c < nout; ++c)
    rowmul[c] = gexp[c] == -100000 ? 0.0f : (gexp[c] - gmax < -126 ? 0.0f : std::ldexp(1.0f, gexp[c] - gmax));
  op.gmax = gmax;
  op.nout = nout;
  op.npad = NOUTP;
  op.K = K;
  op.Kpad = 9 * tpad;
  op.slices = slices;
  op.bits = kBits;
  return RIDG_OK;
}

template <int NB, int NOUTP, bool OUTF2>
static cudaError_t launch_mixed_t(const Grid& g, const double* Q, const MixedOp& op, void* Y,
                                  long long ys_e, long long ys_c, int* texp, int* status,
                                  cudaStream_t s) {
  const MixedLayout L = mixed_layout(op.slices, NB * NB, NOUTP);
  auto kern = predict_mixed_kernel<NB, NOUTP, OUTF2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = ((g.n[0] + kTX - 1) / kTX) * ((g.n[1] + kTY - 1) / kTY);
  const int per_sm = (2 * ((size_t)L.bytes + 2048) <= 233472 && NOUTP <= 32) ? 2 : 1;
  const int grid = std::min(ntiles, sms * per_sm);
  kern<<<grid, kThreads, L.bytes, s>>>(Q, (const uint4*)op.b_slices, op.row_scale, op.row_mul,
                                       op.slices, op.nout, Y, ys_e, ys_c, texp, g.n[0], g.n[1],
                                       status);
  return cudaGetLastError();
}

cudaError_t launch_predict_mixed(const Grid& g, int nb, const double* Q, const MixedOp& op,
                                 double* Y, long long ys_e, long long ys_c, int* status,
                                 cudaStream_t s) {
  if (g.dim != 2) return cudaErrorInvalidValue;
#define RIDG_MIXED_CASE(NBV, NP) \
  case NBV: return launch_mixed_t<NBV, NP, false>(g, Q, op, Y, ys_e, ys_c, nullptr, status, s);
  if (op.npad == 32) {
    switch (nb) { RIDG_MIXED_CASE(2, 32) RIDG_MIXED_CASE(3, 32) RIDG_MIXED_CASE(4, 32) RIDG_MIXED_CASE(5, 32) }
  } else if (op.npad == 64) {
    switch (nb) { RIDG_MIXED_CASE(2, 64) RIDG_MIXED_CASE(3, 64) RIDG_MIXED_CASE(4, 64) RIDG_MIXED_CASE(5, 64) }
  }
#undef RIDG_MIXED_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_predict_fused(const Grid& g, int nb, const double* Q, const MixedOp& op,
                                 void* Y2, int* texp, int* status, cudaStream_t s) {
  if (g.dim != 2) return cudaErrorInvalidValue;
#define RIDG_MIXED_CASE(NBV, NP) \
  case NBV: return launch_mixed_t<NBV, NP, true>(g, Q, op, Y2, 1, g.ncell, texp, status, s);
  if (op.npad == 32) {
    switch (nb) { RIDG_MIXED_CASE(2, 32) RIDG_MIXED_CASE(3, 32) RIDG_MIXED_CASE(4, 32) }
  } else if (op.npad == 64) {
    switch (nb) { RIDG_MIXED_CASE(5, 64) }
  }
#undef RIDG_MIXED_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_correct_fused(const Grid& g, int nb, double* Q, const void* Y2,
                                 const int* texp, int gmax, const CorrParams& cp, int sgnx,
                                 int sgny, cudaStream_t s) {
  if (g.dim != 2) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((g.ncell + 127) / 128);
  const float2* Y = (const float2*)Y2;
#define RIDG_CORR_CASE(NBV)                                                                  \
  case NBV:                                                                                   \
    correct_fused_kernel<NBV><<<blocks, 128, 0, s>>>(Q, Y, texp, g.n[0], g.n[1], cp, gmax,    \
                                                     sgnx, sgny);                             \
    break;
  switch (nb) {
    RIDG_CORR_CASE(2) RIDG_CORR_CASE(3) RIDG_CORR_CASE(4) RIDG_CORR_CASE(5)
    default: return cudaErrorInvalidValue;
  }
#undef RIDG_CORR_CASE
  return cudaGetLastError();
}

size_t mixed_smem_bytes(int nb, const MixedOp& op) {
  return mixed_layout(op.slices, nb * nb, op.npad).bytes;
}

}  // namespace ridg
