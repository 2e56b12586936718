// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits), built from the error-free
// transformations TwoSum (Knuth) and TwoProduct (with a fused multiply-add).
// B300 runs FP64 at a small fraction of its FP32 rate, so the mixed path
// keeps its high-precision intermediates in this form and does its
// element-wise work in FP32 instructions.
#pragma once
#include <cuda_runtime.h>

namespace distil {

// Aligned like float2 / float4 so that arrays of them move with 8- and
// 16-byte accesses (every array of them starts on a 256-byte boundary).
struct __align__(8) DF {
  float hi, lo;
};
struct __align__(16) CDF {  // complex double-float, 16 bytes like complex128
  DF re, im;
};
static_assert(sizeof(DF) == 8 && sizeof(CDF) == 16, "double-float layout");

__device__ __forceinline__ DF df_make(float hi, float lo) { DF r; r.hi = hi; r.lo = lo; return r; }

// s + e = a + b exactly
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ DF quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// p + e = a * b exactly
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df_make(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  const DF t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
// a1 b1 + a2 b2 + a3 b3 + a4 b4 as a double-float: exact products, the
// leading parts summed by TwoSum, the rounding terms added in FP32 (their
// own error is of order 2^-48 of the largest product).
__device__ __forceinline__ DF dot4(float a1, float b1, float a2, float b2, float a3, float b3, float a4, float b4) {
  const float p1 = a1 * b1, p2 = a2 * b2, p3 = a3 * b3, p4 = a4 * b4;
  const float e1 = fmaf(a1, b1, -p1), e2 = fmaf(a2, b2, -p2), e3 = fmaf(a3, b3, -p3), e4 = fmaf(a4, b4, -p4);
  const DF s12 = two_sum(p1, p2), s34 = two_sum(p3, p4);
  const DF s = two_sum(s12.hi, s34.hi);
  const float lo = ((e1 + e2) + (e3 + e4)) + (s12.lo + s34.lo) + s.lo;
  return quick_two_sum(s.hi, lo);
}
// a + b (a - b) with one TwoSum on the leading parts and the trailing parts
// added in FP32: error below 2^-44 (|a| + |b|), enough where the sum is
// not the last word (it feeds products summed in double-float).
__device__ __forceinline__ DF df_add_fast(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_sub_fast(DF a, DF b) {
  const DF s = two_sum(a.hi, -b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo - b.lo));
}
__device__ __forceinline__ DF df_neg(DF a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  DF p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ DF df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return df_make(hi, __double2float_rn(x - (double)hi));
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ CDF cdf_make(DF re, DF im) { CDF c; c.re = re; c.im = im; return c; }
__device__ __forceinline__ CDF cdf_add(CDF a, CDF b) { return cdf_make(df_add(a.re, b.re), df_add(a.im, b.im)); }
__device__ __forceinline__ CDF cdf_scale(CDF a, DF s) { return cdf_make(df_mul(a.re, s), df_mul(a.im, s)); }
__device__ __forceinline__ CDF cdf_conj(CDF a) { return cdf_make(a.re, df_neg(a.im)); }
__device__ __forceinline__ CDF cdf_zero() { return cdf_make(df_make(0.f, 0.f), df_make(0.f, 0.f)); }

}  // namespace distil
