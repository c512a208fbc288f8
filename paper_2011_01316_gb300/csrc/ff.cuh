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
