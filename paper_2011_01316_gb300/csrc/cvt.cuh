// Conversions between IEEE 754 binary32 and binary64 on the integer pipes.
//
// On this GPU the FP64 pipe runs about 1.6 lane operations per SM per clock,
// and cvt.f32.f64 / cvt.f64.f32 issue there too, so a kernel that streams
// FP64 vectors through FP32 arithmetic would be bound by its conversions.
// These functions build the result from the bit fields of the formats
// (binary32: sign, 8-bit exponent with bias 127, 23-bit fraction; binary64:
// sign, 11-bit exponent with bias 1023, 52-bit fraction) with integer and
// logic instructions only:
//
//   f32_to_f64_exact: widening, exact for every input (subnormals included;
//                     NaN payloads kept).
//   f64_to_f32_rn:    narrowing with round-to-nearest-even, overflow to
//                     infinity, gradual underflow to binary32 subnormals;
//                     NaN gives a quiet NaN.
//
// Both are __host__ __device__ so the host tests can compare them with the
// host's own conversions bit for bit.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define EXPDG_HD __host__ __device__ __forceinline__
#else
#define EXPDG_HD inline
#endif

namespace expdg {

EXPDG_HD uint32_t bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
EXPDG_HD float float_of(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
EXPDG_HD void words_of(double x, uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
  hi = (uint32_t)__double2hiint(x);
  lo = (uint32_t)__double2loint(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  hi = (uint32_t)(u >> 32);
  lo = (uint32_t)u;
#endif
}
EXPDG_HD double double_of(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}
EXPDG_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  int n = 0;
  while (n < 32 && !(x & (0x80000000u >> n))) ++n;
  return n;
#endif
}

// Rare paths of the conversions below, out of line so the common (normal
// number) path stays a short straight-line sequence.
#ifdef __CUDACC__
#define EXPDG_COLD static __host__ __device__ __noinline__
#else
#define EXPDG_COLD static inline
#endif

// binary32 -> binary64 of a zero, subnormal, infinity or NaN.
EXPDG_COLD double f32_to_f64_special(uint32_t u) {
  const uint32_t s = u & 0x80000000u, a = u & 0x7fffffffu;
  uint32_t hi, lo;
  if (a >= 0x7f800000u) {  // infinity or NaN: all-ones exponent
    hi = s | ((a >> 3) + 0x70000000u);
    lo = a << 29;
  } else if (a == 0u) {
    hi = s;
    lo = 0u;
  } else {  // subnormal m 2^-149: normalise m to a leading one at bit 23
    const int sh = clz32(a) - 8;
    const uint32_t mant = (a << sh) & 0x007fffffu;
    hi = s | ((uint32_t)(897 - sh) << 20) | (mant >> 3);
    lo = mant << 29;
  }
  return double_of(hi, lo);
}

// binary32 -> binary64, exact.
EXPDG_HD double f32_to_f64_exact(float x) {
  const uint32_t u = bits_of(x);
  const uint32_t a = u & 0x7fffffffu;
  if (a - 0x00800000u >= 0x7f000000u) return f32_to_f64_special(u);
  // normal: exponent field + (1023 - 127) in the binary64 position, fraction split 20 / 3
  return double_of((u & 0x80000000u) | ((a >> 3) + 0x38000000u), a << 29);
}

// binary64 -> binary32 (round to nearest, ties to even) of a value outside the
// binary32 normal range: infinity, NaN, overflow, subnormal results, zero.
EXPDG_COLD float f64_to_f32_special(uint32_t hi, uint32_t lo) {
  const uint32_t s = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
  if (ahi >= 0x7ff00000u) {  // infinity or NaN
    const bool nan = (ahi & 0x000fffffu) != 0u || lo != 0u;
    return float_of(s | (nan ? 0x7fc00000u : 0x7f800000u));
  }
  if (ahi >= 0x47f00000u) return float_of(s | 0x7f800000u);  // >= 2^128: overflow
  // below the binary32 normal range: m_f = round(significand 2^(e - 926))
  const int e = (int)(ahi >> 20);
  const int sh = 926 - e;  // >= 30
  if (e == 0 || sh > 54) return float_of(s);  // rounds to zero
  const uint64_t fm = ((uint64_t)(ahi & 0x000fffffu) << 32 | lo) | ((uint64_t)1 << 52);
  uint64_t q = fm >> sh;
  const uint64_t rem = fm & (((uint64_t)1 << sh) - 1), half = (uint64_t)1 << (sh - 1);
  if (rem > half || (rem == half && (q & 1u))) q += 1u;  // q = 2^23 is the smallest normal: correct
  return float_of(s | (uint32_t)q);
}

// binary64 -> binary32, round to nearest, ties to even.
EXPDG_HD float f64_to_f32_rn(double x) {
  uint32_t hi, lo;
  words_of(x, hi, lo);
  const uint32_t ahi = hi & 0x7fffffffu;
  if (ahi - 0x38100000u >= 0x0fe00000u) return f64_to_f32_special(hi, lo);
  // binary64 exponent 897..1150, a normal binary32 result:
  // (e - 896) << 23 | top 23 fraction bits; the 29 bits below decide the rounding
  uint32_t r = ((ahi - 0x38000000u) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry may reach infinity: correct
  return float_of((hi & 0x80000000u) | r);
}

}  // namespace expdg
