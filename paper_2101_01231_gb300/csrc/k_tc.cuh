// Shared device helpers of the tensor-core (tcgen05 + TMA) kernels of the mixed linear path:
// shared-memory matrix descriptors, the BF16 MMA, bounded mbarrier waits, TMA and bulk
// copies, TMEM loads, error-free FP32 sums, and the split of FP64 coefficients into balanced
// base-256 digits (exact in BF16).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ridg {
namespace {

constexpr int kTX = 8, kTY = 16;             // cells per tile in x, y (128 = MMA M)
constexpr int kHX = kTX + 2, kHY = kTY + 2;  // halo
constexpr int kCopy = kTX * kHY;             // cells of one x-shifted halo copy (8 x 18)
constexpr int kBits = 8;                     // digit width
constexpr long kWaitLimit = 1L << 22;        // bounded mbarrier polls (well under a second)
constexpr int kGemmThreads = 320;            // warp 0: TMA, warp 1: MMA, warps 2..9: epilogue
constexpr int kMaxSlots = 8;                 // ring of per-digit operand slots
constexpr uint32_t kSmemLimit = 232448;      // opt-in shared memory per block

// status bits
constexpr int kStatusTimeout = 2;
constexpr int kStatusRange = 4;

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

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
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

// the same bounded wait with a short sleep between polls (for warps that only consume)
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (!done) __nanosleep(64);
  }
  return done != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%6];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(0), "r"(mbar)
      : "memory");
}

// bring a TMA box into L2 ahead of its load (no shared memory, no barrier)
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   (uint64_t)map),
               "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

// 8 consecutive TMEM columns of this thread's lane (no wait: see tmem_wait_ld)
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
  if (ex == 0) return 0;  // zero / subnormal: far below the state's scale
  const long long mant = (long long)((u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = ex - 1075 + L - s;
  long long F;
  if (sh >= 0) {
    F = sh < 11 ? (mant << sh) : (1LL << 62);  // out of range: flagged by the caller
  } else if (sh > -63) {
    F = (mant + (1LL << (-sh - 1))) >> (-sh);
  } else {
    F = 0;
  }
  return (u >> 63) ? -F : F;
}

// S balanced base-256 digits of 8 consecutive coefficients, packed as BF16 (one 16 B row
// per digit).  Returns false if a value does not fit below 2^s.
template <int S>
__device__ __forceinline__ bool make_digit_rows(const double* v, int s, uint4* rows) {
  constexpr int L = kBits * S;
  uint32_t packed[S][4];
  bool fits = true;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long F = to_fixed(v[j], s, L);
    fits &= (F < (1LL << L)) && (F > -(1LL << L));
    const uint32_t lo32 = (uint32_t)F, hi32 = (uint32_t)((unsigned long long)F >> 32);
    const int neg = (int)(hi32 >> 31);
    int carry = 0;
    int d[S];
#pragma unroll
    for (int a = S - 1; a >= 0; --a) {
      const int k = S - 1 - a;  // byte index of digit a
      const uint32_t byte = (k < 4 ? (lo32 >> (8 * k)) : (hi32 >> (8 * (k - 4)))) & 0xFFu;
      if (a > 0) {
        const int t = (int)byte + carry;
        carry = (t + 128) >> 8;
        d[a] = t - (carry << 8);
      } else {
        d[0] = (int)byte - (neg << 8) + carry;
      }
    }
#pragma unroll
    for (int a = 0; a < S; ++a) {
      // |d| <= 256: exact in FP32 by the 1.5 * 2^23 trick, and its BF16 is the top half
      const uint32_t b = __float_as_uint(__int_as_float(0x4B400000 + d[a]) - 12582912.0f) >> 16;
      if (j & 1)
        packed[a][j / 2] |= b << 16;
      else
        packed[a][j / 2] = b;
    }
  }
#pragma unroll
  for (int a = 0; a < S; ++a) rows[a] = make_uint4(packed[a][0], packed[a][1], packed[a][2], packed[a][3]);
  return fits;
}

__device__ __forceinline__ int exponent_above(unsigned long long absbits) {
  // e with max < 2^e (0 for a zero maximum)
  return absbits == 0 ? 0 : (int)((absbits >> 52) & 0x7FF) - 1022;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v,
                                                             unsigned long long* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = sh[w] > r ? sh[w] : r;
  return r;
}

// max |q| of the state -> maxbits[1]
__global__ void state_max_kernel(const double* __restrict__ q, long long count,
                                 unsigned long long* maxbits) {
  __shared__ unsigned long long sh[8];
  unsigned long long m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(q[i]) & 0x7FFFFFFFFFFFFFFFULL;
    m = a > m ? a : m;
  }
  m = block_max_bits(m, sh);
  if (threadIdx.x == 0) atomicMax(maxbits + 1, m);
}

}  // namespace
}  // namespace ridg
