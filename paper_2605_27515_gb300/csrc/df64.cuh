// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// (about 48 bits of significand, the exponent range of float).  On GB300 the FP32
// pipes issue 64 times as many operations per clock as the FP64 pipe, so a
// double-float operation built from a handful of FP32 instructions is several
// times faster than native FP64 while keeping ~1e-14 relative accuracy.
//
// The building blocks are the classical error-free transformations: Knuth's
// two-sum (the rounding error of a + b, exactly) and the fused-multiply-add
// product (the rounding error of a * b is fma(a, b, -a*b), exactly), followed by
// renormalisation so that |lo| <= ulp(hi) / 2.
#pragma once

#include <cuda_runtime.h>

namespace qlb {

struct df64 {
  float hi, lo;
  __host__ __device__ __forceinline__ df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ df64(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ __forceinline__ df64(int x) : df64((double)x) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, given |a| >= |b|
__device__ __forceinline__ void df_quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e, t, f;
  df_two_sum(a.hi, b.hi, s, e);
  df_two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  df_quick_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  df64 r;
  df_quick_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df64 r;
  df_quick_two_sum(p, e, r.hi, r.lo);
  return r;
}
// c + a * b with one renormalisation (the product's error terms and the sum's
// rounding error folded into the low word): the multiply-add of the GEMM
__device__ __forceinline__ df64 df_mac(df64 c, df64 a, df64 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, e;
  df_two_sum(c.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(c.lo, pe));
  df64 r;
  df_quick_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  // long division: q1 = a/b in float, remainder in double-float, one correction
  float q1 = a.hi / b.hi;
  df64 r = a - b * df64(q1, 0.f);
  float q2 = r.hi / b.hi;
  df64 q;
  df_quick_two_sum(q1, q2, q.hi, q.lo);
  return q;
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return b > a; }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(b > a); }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(a > b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ df64 sqrt(df64 a) {
  // one Newton step on the float square root: x + (a - x^2) / (2x)
  if (!(a.hi > 0.f)) return df64(0.f, 0.f);
  float x = sqrtf(a.hi);
  df64 xx = df64(x, 0.f);
  df64 r = a - xx * xx;
  float corr = r.hi / (2.f * x);
  df64 out;
  df_quick_two_sum(x, corr, out.hi, out.lo);
  return out;
}
__device__ __forceinline__ bool isfinite(df64 a) { return ::isfinite(a.hi); }
// keep the double versions visible next to the overloads above
__device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
__device__ __forceinline__ bool isfinite(double x) { return ::isfinite(x); }
__host__ __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

}  // namespace qlb
