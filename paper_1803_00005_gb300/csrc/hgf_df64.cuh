// Double-float arithmetic: a value is the unevaluated sum hi + lo of two float32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits. It stands in for float64 in the guidance
// inverse, where GB300 runs float32 at 64 times the float64 rate. The algorithms are the
// published error-free transformations and double-word operations:
//   two_sum (Knuth, TAOCP vol. 2, 1969), fast_two_sum (Dekker, Numer. Math. 18, 1971),
//   two_prod via one fused multiply-add, and the double-word addition, multiplication and
//   division of Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic building
//   blocks of double-word arithmetic", ACM TOMS 44(2), 2017 (Algorithms 6, 12 and 18 there).
// Only + - * / and fmaf are used; no library math function is reimplemented. Host code never
// sees this type.
#pragma once

namespace hgf {

struct df64 {
  float hi, lo;
  __device__ __forceinline__ df64() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64(float f) : hi(f), lo(0.f) {}
  __device__ __forceinline__ explicit df64(int i) {
    hi = (float)i;  // exact for |i| < 2^24
    lo = (float)(i - (int)hi);
  }
  __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df64(s, e);
}
// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return df64(s, e);
}
// p + e = a * b exactly
__device__ __forceinline__ df64 two_prod(float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  return df64(p, e);
}

// double-word + double-word (accurate version)
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  df64 s = two_sum(x.hi, y.hi);
  const df64 t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

// double-word * double-word
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  df64 p = two_prod(x.hi, y.hi);
  const float t = fmaf(x.lo, y.hi, x.hi * y.lo);
  p.lo += t;
  return fast_two_sum(p.hi, p.lo);
}

// double-word / double-word: a float32 quotient of the leading words, then one correction
// from the double-word remainder
__device__ __forceinline__ df64 operator/(df64 x, df64 y) {
  const float q1 = x.hi / y.hi;
  const df64 r = x - y * df64(q1);
  const float q2 = r.hi / y.hi;
  return fast_two_sum(q1, q2);
}

// a * b + c with the double-word operations above
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }

}  // namespace hgf
