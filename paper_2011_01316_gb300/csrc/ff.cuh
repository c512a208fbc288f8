// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// h + l of two FP32 numbers with |l| <= ulp(h)/2, a 48-bit significand.
//
// Error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and the
// FMA-based TwoProduct (as in Ogita, Rump & Oishi, "Accurate sum and dot
// product", SISC 2005).  Every operation is written with the _rn intrinsics,
// which the compiler never contracts into FMAs, so the transformations stay
// exact.  All arithmetic is FP32 (the FFMA pipe), never the FP64 pipe.
#pragma once
#include <cuda_runtime.h>

namespace expdg {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return ff_fast_two_sum(s.h, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }

// exact product of two floats as a float-float
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return ff_fast_two_sum(p, e);
}

// acc + a * b
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff acc) {
  float p = __fmul_rn(a.h, b.h);
  float pe = __fmaf_rn(a.h, b.h, -p);
  pe = __fmaf_rn(a.h, b.l, pe);
  pe = __fmaf_rn(a.l, b.h, pe);
  ff s = ff_two_sum(acc.h, p);
  float e = __fadd_rn(s.l, __fadd_rn(pe, acc.l));
  return ff_fast_two_sum(s.h, e);
}

// Conversions touch the FP64 pipe; use them only outside streaming loops.
__device__ __forceinline__ ff ff_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ff ff_shfl_down(ff a, int off) {
  return {__shfl_down_sync(0xffffffffu, a.h, off), __shfl_down_sync(0xffffffffu, a.l, off)};
}

}  // namespace expdg

namespace expdg {

// ---- two lanes at once (Blackwell packed FP32: FADD2 / FMUL2 / FFMA2) ----
// These halve the instruction count of the error-free transformations; the
// FP32 pipe itself runs one lane-operation per lane per clock either way.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Compensated dot-product accumulation (the Dot2 scheme of Ogita, Rump & Oishi,
// with float-float operands): S carries the running sum of the rounded
// products (TwoSum keeps it exact), C the product errors (TwoProduct), the
// low-part cross terms and the TwoSum errors.  12 packed instructions per two
// terms.  The value of the sum is S + C.
__device__ __forceinline__ void dot2_acc(float2 xh, float2 xl, float2 yh, float2 yl, float2& S, float2& C) {
  const float2 p = mul2(xh, yh);
  float2 e = fma2(xh, yh, neg2(p));
  e = fma2(xh, yl, e);
  e = fma2(xl, yh, e);
  const float2 s = add2(S, p);
  const float2 bb = sub2(s, S);
  const float2 err = add2(sub2(S, sub2(s, bb)), sub2(p, bb));
  S = s;
  C = add2(C, add2(err, e));
}

// x += c * q with x = (xh, xl) kept un-normalised: xh takes the rounded
// products exactly (TwoSum), xl collects every error term.  Normalise with
// ff2_norm after at most a few dozen terms.
__device__ __forceinline__ void axpy2_acc(float2 ch, float2 cl, float2 qh, float2 ql, float2& xh, float2& xl) {
  const float2 p = mul2(ch, qh);
  float2 e = fma2(ch, qh, neg2(p));
  e = fma2(ch, ql, e);
  e = fma2(cl, qh, e);
  const float2 s = add2(xh, p);
  const float2 bb = sub2(s, xh);
  const float2 err = add2(sub2(xh, sub2(s, bb)), sub2(p, bb));
  xh = s;
  xl = add2(xl, add2(err, e));
}

// (h, l) <- TwoSum(h, l): exact renormalisation whatever the magnitudes
// (after cancellation |l| may exceed |h|).
__device__ __forceinline__ void ff2_norm(float2& h, float2& l) {
  const float2 s = add2(h, l);
  const float2 bb = sub2(s, h);
  const float2 e = add2(sub2(h, sub2(s, bb)), sub2(l, bb));
  h = s;
  l = e;
}

// (h, l) * c for a float-float scalar c, result normalised (|e| << |p|).
__device__ __forceinline__ void ff2_scale(float2& h, float2& l, float2 ch, float2 cl) {
  const float2 p = mul2(h, ch);
  float2 e = fma2(h, ch, neg2(p));
  e = fma2(h, cl, e);
  e = fma2(l, ch, e);
  const float2 s2 = add2(p, e);
  l = sub2(e, sub2(s2, p));
  h = s2;
}

// S + C of dot2_acc, both lanes summed, as one float-float value.
__device__ __forceinline__ ff dot2_value(float2 S, float2 C) {
  ff t = ff_two_sum(S.x, S.y);
  const float c = __fadd_rn(__fadd_rn(C.x, C.y), t.l);
  return ff_fast_two_sum(t.h, c);
}

}  // namespace expdg
