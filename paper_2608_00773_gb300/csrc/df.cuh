// Double-float arithmetic (a value is hi + lo, two FP32 numbers with
// |lo| <= ulp(hi)/2): about 44 significant bits on the FP32 pipes.
// Error-free transformations after Dekker (1971) and Knuth (TAOCP vol. 2):
// two-sum, fast two-sum and the FMA two-product.  Every step uses the _rn
// intrinsics so that no multiply-add is contracted into a fused one.
#pragma once

#include <cstdint>

namespace q4c {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h) { return {h, 0.0f}; }

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df x, float f) {
  const float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return fast_two_sum(p, e);
}

// x * y + z
__device__ __forceinline__ df df_fma(df x, df y, df z) { return df_add(df_mul(x, y), z); }

// x / y: one FP32 quotient and one correction step
__device__ __forceinline__ df df_div(df x, df y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const df r = df_sub(x, df_mul_f(y, q1));
  const float q2 = __fdiv_rn(r.hi, y.hi);
  return fast_two_sum(q1, q2);
}

// sqrt(x), x > 0: FP32 root and one Newton correction
__device__ __forceinline__ df df_sqrt(df x) {
  const float s = __fsqrt_rn(x.hi);
  const df ss = df_mul(df_make(s), df_make(s));
  const df r = df_sub(x, ss);
  const float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
  return fast_two_sum(s, c);
}

}  // namespace q4c
