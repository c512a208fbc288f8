// fx: a float-float number (h + l, 48-bit significand) with arithmetic
// operators, so the DG operator templates can run in float-float on the FP32
// pipes (the mixed form's residual).  Built on the error-free transformations
// of ff.cuh; division and square root take the FP32 quotient / root and one
// Newton correction in float-float (Dekker's method), accurate to a few units
// of 2^-48.
#pragma once
#include "ff.cuh"

namespace expdg {

// the float / double overloads stay visible next to the float-float ones below
using ::fabs;
using ::fmax;
using ::sqrt;

struct fx {
  float h, l;
  fx() = default;
  __device__ __forceinline__ constexpr fx(float hh, float ll) : h(hh), l(ll) {}
  __device__ __forceinline__ explicit fx(float f) : h(f), l(0.0f) {}
  __device__ __forceinline__ explicit fx(int i) : fx((double)i) {}
  // rounding split of a double; for literal constants the compiler folds it
  __device__ __forceinline__ explicit fx(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  __device__ __forceinline__ fx(ff a) : h(a.h), l(a.l) {}
  __device__ __forceinline__ operator ff() const { return ff{h, l}; }
};

__device__ __forceinline__ fx operator+(fx a, fx b) { return ff_add(a, b); }
__device__ __forceinline__ fx operator-(fx a) { return fx(-a.h, -a.l); }
__device__ __forceinline__ fx operator-(fx a, fx b) { return ff_add(a, ff{-b.h, -b.l}); }
__device__ __forceinline__ fx operator*(fx a, fx b) { return ff_mul(a, b); }
__device__ __forceinline__ fx operator/(fx a, fx b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const fx r = a - b * fx(q1);  // remainder, exact up to float-float rounding
  const float q2 = __fdiv_rn(r.h, b.h);
  return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ fx& operator+=(fx& a, fx b) { return a = a + b; }
__device__ __forceinline__ fx& operator-=(fx& a, fx b) { return a = a - b; }
__device__ __forceinline__ fx& operator*=(fx& a, fx b) { return a = a * b; }

__device__ __forceinline__ bool operator<(fx a, fx b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ bool operator>(fx a, fx b) { return b < a; }
__device__ __forceinline__ bool operator<=(fx a, fx b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(fx a, fx b) { return !(a < b); }

__device__ __forceinline__ fx fabs(fx a) { return (a.h < 0.0f || (a.h == 0.0f && a.l < 0.0f)) ? -a : a; }
__device__ __forceinline__ fx fmax(fx a, fx b) { return (a < b) ? b : a; }
__device__ __forceinline__ fx sqrt(fx a) {
  if (!(a.h > 0.0f)) return fx(__fsqrt_rn(a.h), 0.0f);  // 0, or NaN for a negative argument
  const float s = __fsqrt_rn(a.h);
  const fx e = a - fx(ff_two_prod(s, s));  // a - s^2
  return ff_fast_two_sum(s, __fdiv_rn(e.h, 2.0f * s));
}

}  // namespace expdg
