// Products of a double and a small integer, rounded to nearest even, by integer operations on the
// bit pattern.  The three-term recursions for Delta multiply every step's coefficient a(m') by the
// column's 2m; on this part the FP64 pipe does 2 operations per SM and clock against 64 or more for
// the integer pipe, so this product moves there and an update keeps two FP64 instructions (the
// product with the previous value and the fused multiply-add).  Plain C++ as well, so that the
// CPU tests compile this same code and compare it with IEEE multiplication.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define SSHT_HD __host__ __device__ __forceinline__
#else
#define SSHT_HD inline
#endif

namespace ssht {

SSHT_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// Bit pattern of fl(k x 2^d): the double nearest to k x 2^d, ties to even, for an integer
// 0 <= k < 2^11, a double x >= 0 that is zero or normal, and a small d >= 0 such that the result
// stays below 2^1024.  With x = M 2^(e - 1075) (M the 53-bit significand, implicit bit set; e the
// biased exponent) the product P = k M is exact in 64 bits (M < 2^53, k < 2^11).  If P has
// 53 + s bits, its s low bits are rounded off -- adding 2^(s-1) - 1 plus the lowest kept bit and
// truncating rounds to nearest with ties to even -- and the exponent grows by s.  A rounding that
// carries out of 53 bits (R = 2^53) lands in the exponent field through the addition that
// assembles the result, as it must.
SSHT_HD uint64_t mul_small_rn_bits(uint64_t xb, uint32_t k, int d) {
  if (xb == 0 || k == 0) return 0;
  const uint64_t M = (xb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const uint64_t e = xb >> 52;
  const uint64_t P = M * (uint64_t)k;
  const int s = 11 - clz64(P);  // P >= 2^52, so 0 <= s <= 11
  const uint64_t mask = (1ull << s) - 1ull, half = (1ull << s) >> 1;
  const uint64_t R = (P + ((half - 1ull + ((P >> s) & 1ull)) & mask)) >> s;
  return ((e + (uint64_t)(s + d)) << 52) + R - 0x0010000000000000ull;
}

#if defined(__CUDACC__)
__device__ __forceinline__ double mul_small_rn(double x, uint32_t k, int d) {
  return __longlong_as_double((long long)mul_small_rn_bits((uint64_t)__double_as_longlong(x), k, d));
}
#endif

}  // namespace ssht
