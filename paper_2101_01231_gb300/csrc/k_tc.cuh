// Shared device helpers of the tensor-core (tcgen05 + TMA) kernels of the mixed linear path:
// tile constants, TMA tensor copies, error-free FP32 sums, and the split of FP64 coefficients
// into balanced base-256 digits (exact in BF16).  The tcgen05 / mbarrier / bulk-copy wrappers
// are in k_tcgen05.cuh.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "k_tcgen05.cuh"

namespace ridg {
namespace {

constexpr int kTX = 8, kTY = 16;             // cells per tile in x, y (128 = MMA M)
constexpr int kHX = kTX + 2, kHY = kTY + 2;  // halo
constexpr int kCopy = kTX * kHY;             // cells of one x-shifted halo copy (8 x 18)
constexpr int kBits = 8;                     // digit width
constexpr int kGemmThreads = 320;            // warp 0: TMA, warp 1: MMA, warps 2..9: epilogue
constexpr int kMaxSlots = 8;                 // ring of per-digit operand slots
constexpr uint32_t kSmemLimit = 232448;      // opt-in shared memory per block

// status bits
constexpr int kStatusTimeout = 2;
constexpr int kStatusRange = 4;

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

// The same for L <= 24 fraction bits, in 32-bit arithmetic: F = round-half-up(|x| 2^(L - s))
// with x's sign, |F| < 2^L (returns false, F = 0, where it is not).  With the 53-bit
// significand m and sh = 1075 - e - L + s, F = (t + 1) >> 1 for t = floor(m / 2^(sh - 1)) --
// the same value as (m + 2^(sh - 1)) >> sh; t is below 2^32 only for sh - 1 >= 21, and
// F < 2^L needs more than that, so smaller shifts are out of range.
template <int L>
__device__ __forceinline__ bool to_fixed32(double x, int s, int& F) {
  static_assert(L <= 24, "32-bit fixed point");
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  F = 0;
  if (ex == 0) return true;  // zero / subnormal: far below the state's scale
  const int r = 1074 - ex - L + s;  // sh - 1
  if (r < 21) return false;         // |x| 2^(L - s) >= 2^31 (or not finite)
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;  // the significand's top 21 bits
  const uint32_t t = r < 32 ? __funnelshift_r(lo, mh, r) : (r < 53 ? mh >> (r - 32) : 0u);
  const uint32_t f = (t + 1u) >> 1;
  if (f >= (1u << L)) return false;
  F = (hi >> 31) ? -(int)f : (int)f;
  return true;
}

// The same for 24 < L <= 52 fraction bits (|F| < 2^L in 64 bits): t = floor(m / 2^(sh - 1))
// by funnel shifts of the significand's two words, F = (t + 1) >> 1.  Shifts below 0 are out
// of range (|x| 2^(L - s) >= 2^52 >= 2^L).
template <int L>
__device__ __forceinline__ bool to_fixed64(double x, int s, long long& F) {
  static_assert(L > 24 && L <= 52, "64-bit fixed point below the significand's width");
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  F = 0;
  if (ex == 0) return true;  // zero / subnormal: far below the state's scale
  const int r = 1074 - ex - L + s;  // sh - 1
  if (r < 0) return false;
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
  uint32_t tl, th;
  if (r < 32) {
    tl = __funnelshift_r(lo, mh, r);
    th = mh >> r;
  } else {
    tl = r < 53 ? mh >> (r - 32) : 0u;
    th = 0u;
  }
  const unsigned long long t = ((unsigned long long)th << 32) | tl;
  const unsigned long long f = (t + 1ull) >> 1;
  if (f >= (1ull << L)) return false;
  F = (hi >> 31) ? -(long long)f : (long long)f;
  return true;
}

// The S balanced base-256 digits of one coefficient (fixed point with 8 S fraction bits
// relative to 2^s), most significant first, as BF16 (or, f16, FP16) bit patterns (exact
// either way: |digit| <= 256).  Returns false if the value does not fit below 2^s.
template <int S>
__device__ __forceinline__ bool value_digit_bits(double x, int s, uint32_t (&bits)[S],
                                                 bool f16 = false) {
  constexpr int L = kBits * S;
  bool fits;
  int d[S];
  if constexpr (L <= 24) {
    // 32-bit: with 128 added at every lower digit position, the lower digits are the bytes
    // minus 128 and the top digit is the arithmetic shift (the same balanced digits as the
    // carry loop below)
    int F;
    fits = to_fixed32<L>(x, s, F);
    constexpr int kOff = S == 3 ? 0x8080 : (S == 2 ? 0x80 : 0);
    const int G = F + kOff;
#pragma unroll
    for (int a = S - 1; a > 0; --a) d[a] = ((G >> (8 * (S - 1 - a))) & 0xFF) - 128;
    d[0] = G >> (8 * (S - 1));
  } else {
    // 64-bit, the same offset (128 at each of the S - 1 lower digit positions)
    long long F;
    if constexpr (L <= 52) {
      fits = to_fixed64<L>(x, s, F);
    } else {
      F = to_fixed(x, s, L);
      fits = (F < (1LL << L)) && (F > -(1LL << L));
    }
    unsigned long long off = 0;
#pragma unroll
    for (int k = 0; k < S - 1; ++k) off |= 0x80ull << (8 * k);
    const long long G = F + (long long)off;
    const uint32_t g0 = (uint32_t)G, g1 = (uint32_t)((unsigned long long)G >> 32);
#pragma unroll
    for (int a = S - 1; a > 0; --a) {
      const int k = S - 1 - a;  // byte index of digit a
      d[a] = (int)((k < 4 ? (g0 >> (8 * k)) : (g1 >> (8 * (k - 4)))) & 0xFFu) - 128;
    }
    d[0] = (int)(G >> (8 * (S - 1)));
  }
#pragma unroll
  for (int a = 0; a < S; ++a)
    // |d| <= 256: exact in FP32 by the 1.5 * 2^23 trick; its BF16 is the top half, its FP16
    // the exact conversion
    bits[a] = f16 ? (uint32_t)__half_as_ushort(__int2half_rn(d[a]))
                  : __float_as_uint(__int_as_float(0x4B400000 + d[a]) - 12582912.0f) >> 16;
  return fits;
}

// S balanced base-256 digits of 8 consecutive coefficients, packed as BF16 (one 16 B row
// per digit).  Returns false if a value does not fit below 2^s.
template <int S>
__device__ __forceinline__ bool make_digit_rows(const double* v, int s, uint4* rows,
                                                bool f16 = false) {
  uint32_t packed[S][4];
  bool fits = true;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint32_t b[S];
    fits &= value_digit_bits<S>(v[j], s, b, f16);
#pragma unroll
    for (int a = 0; a < S; ++a) {
      if (j & 1)
        packed[a][j / 2] |= b[a] << 16;
      else
        packed[a][j / 2] = b[a];
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
