// FP64 -> FP32 conversion, round to nearest even, by integer operations on the bit pattern (the
// FP64 pipe, where a conversion instruction would run, is the scarce one on this part).  Shared
// by the operand packing and the recursion's tile output; plain C++ as well, so that the CPU tests
// compile this same code and compare it with IEEE rounding.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define SSHT_HD __host__ __device__ __forceinline__
#else
#define SSHT_HD inline
#endif

namespace ssht {

// Bit pattern of the FP32 value nearest to the double with bit pattern b (ties to even), for
// |x| < 2^128 (larger magnitudes are not produced here: every converted value is below 20).
// Normal range: adding 2^28 - 1 plus the lowest kept bit rounds the 29 dropped fraction bits, a
// carry moving into the exponent as rounding requires, and the exponent is rebiased from 1023 to
// 127.  Below 2^-126 the result is an FP32 subnormal: the 53-bit significand is shifted right so
// that its unit is 2^-149 and rounded to nearest even; below 2^-150 the result is a signed zero
// (2^-150 itself is a tie and goes to the even zero).
SSHT_HD uint32_t f64_bits_to_f32_rn(uint64_t b) {
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int ef = (int)((b >> 52) & 0x7FF);  // biased FP64 exponent
  if (ef > 896) {
    const uint64_t t = b + 0x0FFFFFFFull + ((b >> 29) & 1u);
    return sign | (((uint32_t)(t >> 29) - (896u << 23)) & 0x7FFFFFFFu);
  }
  // |x| < 2^-126: value = mant * 2^(ef - 1075) with the implicit bit (ef >= 1); in units of 2^-149
  // that is mant >> (926 - ef)
  const int shift = 926 - ef;
  if (ef == 0 || shift > 53) return sign;
  const uint64_t mant = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const uint64_t q = mant >> shift;
  const uint64_t rem = mant & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
  const uint64_t r = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
  return sign | (uint32_t)r;  // r = 2^23 is the smallest normal, encoded by the same bits
}

#if defined(__CUDACC__)
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  return __uint_as_float(f64_bits_to_f32_rn((uint64_t)__double_as_longlong(x)));
}
#endif

}  // namespace ssht
