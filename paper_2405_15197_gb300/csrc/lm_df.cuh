// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// The FP64 stability steps of the meta-mesh build (candidate vertices whose
// FP32 screening is inside a margin) only need +, -, *, / and sqrt, and their
// thresholds sit at 1e-9 R or coarser, far above the ~1e-14 relative error of
// this format.  On GB300 an FP64 instruction costs 64x the FP32 issue rate,
// so these steps run in double-float on the FP32 pipes instead.
//
// Building blocks (error-free transformations):
//  * two_sum (Knuth): s = fl(a + b) and e with a + b = s + e exactly;
//  * fast_two_sum (Dekker), valid when |a| >= |b|;
//  * two_prod with a fused multiply-add: p = fl(a b), e = fma(a, b, -p).
// The operators below combine them in the usual way: add and subtract carry
// both error terms, multiply adds the cross terms, divide and sqrt take one
// FP32 estimate and one Newton correction computed in double-float.
#pragma once
#include <cuda_runtime.h>

namespace lm {

// the overloads below join, not hide, the FP32/FP64 ones
using ::fabs;
using ::fmax;
using ::fmin;

struct df {
  float hi, lo;
  __host__ __device__ df() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df(float x) : hi(x), lo(0.0f) {}
  __host__ __device__ df(int x) : hi((float)x), lo((float)(x - (int)(float)x)) {}
  __host__ __device__ df(bool x) : hi(x ? 1.0f : 0.0f), lo(0.0f) {}
  __host__ __device__ explicit df(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df(s, e);
}
__device__ __forceinline__ df df_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return df(p, e);
}

__device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  df t = df_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  df p = df_two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df operator/(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = a - b * df(q1);
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = r - b * df(q2);
  float q3 = __fdiv_rn(r.hi, b.hi);
  df q = df_fast_two_sum(q1, q2);
  return q + df(q3);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }

__device__ __forceinline__ df fabs(df a) { return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? -a : a; }
__device__ __forceinline__ df fmax(df a, df b) { return a < b ? b : a; }
__device__ __forceinline__ df fmin(df a, df b) { return b < a ? b : a; }

// square root: FP32 estimate s, then s + (a - s^2) / (2 s) in double-float
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.0f)) return df(0.0f);
  float s = __fsqrt_rn(a.hi);
  df s2 = df_two_prod(s, s);
  df r = a - s2;
  float c = __fdiv_rn(r.hi, 2.0f * s);
  return df_fast_two_sum(s, c);
}

}  // namespace lm
