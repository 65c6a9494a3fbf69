// Double-float arithmetic: a value is the unevaluated sum hi + lo of two float32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits. It stands in for float64 in the guidance
// inverse, where GB300 runs float32 at 64 times the float64 rate. The algorithms are the
// published error-free transformations and double-word operations:
//   two_sum (Knuth, TAOCP vol. 2, 1969), fast_two_sum (Dekker, Numer. Math. 18, 1971),
//   two_prod via one fused multiply-add, and the double-word addition, multiplication and
//   division of Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic building
//   blocks of double-word arithmetic", ACM TOMS 44(2), 2017 (Algorithms 6, 12 and 18 there).
// The transformations are only error-free when every rounding happens as written, so the sums
// and products go through the round-to-nearest intrinsics __fadd_rn / __fsub_rn / __fmul_rn,
// which the compiler never contracts into fused multiply-adds (a contracted a*b + c would
// break the exactness of two_sum and fast_two_sum). float64 is used only to split a float64
// input once; no library math function is reimplemented. Host code never sees this type.
#pragma once

namespace hgf {
// in a namespace of its own so that the overloads below (fma, sqrt) are found by argument-
// dependent lookup for df64 only and do not hide the float and double ones
namespace dw {

struct df64 {
  float hi, lo;
  __device__ __forceinline__ df64() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64(float f) : hi(f), lo(0.f) {}
  __device__ __forceinline__ explicit df64(int i) {
    hi = (float)i;  // exact for |i| < 2^24
    lo = (float)(i - (int)hi);
  }
  __device__ __forceinline__ explicit df64(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}
// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df64(s, e);
}
// p + e = a * b exactly
__device__ __forceinline__ df64 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  return df64(p, e);
}

// double-word + double-word (accurate version)
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  df64 s = two_sum(x.hi, y.hi);
  const df64 t = two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

// double-word * double-word
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  df64 p = two_prod(x.hi, y.hi);
  const float t = fmaf(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
  p.lo = __fadd_rn(p.lo, t);
  return fast_two_sum(p.hi, p.lo);
}

// double-word / double-word: a float32 quotient of the leading words, then one correction
// from the double-word remainder
__device__ __forceinline__ df64 operator/(df64 x, df64 y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const df64 r = x - y * df64(q1);
  const float q2 = __fdiv_rn(r.hi, y.hi);
  return fast_two_sum(q1, q2);
}

// a * b + c with the double-word operations above
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ df64 &operator+=(df64 &x, df64 y) { return x = x + y; }

// square root: the float32 root of the leading word, then one Newton step with the exact
// double-word remainder x - s1^2 (the refinement of Hida, Li and Bailey, "Algorithms for
// quad-double precision floating point arithmetic", ARITH 15, 2001); x >= 0
__device__ __forceinline__ df64 sqrt(df64 x) {
  if (!(x.hi > 0.f)) return df64(0.f, 0.f);
  const float s1 = __fsqrt_rn(x.hi);
  const df64 r = x - two_prod(s1, s1);
  const float s2 = __fdiv_rn(r.hi, __fmul_rn(2.f, s1));
  return fast_two_sum(s1, s2);
}

}  // namespace dw
using dw::df64;
}  // namespace hgf
