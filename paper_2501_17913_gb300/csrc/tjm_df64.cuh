// FP64 emulation on the FP32 pipes: double-float ("double-word") numbers.
//
// A df64 value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, i.e. a 48-bit significand with the FP32 exponent range.
// GB300 issues 2 FP64 FMAs per clock per SM against 128 FP32 FMAs, so the
// factorizations that the precision plan keeps in FP64 (QR, SVD) run here in
// this representation: about 20 FP32 instructions per df64 multiply-add, a
// third of the issue cost of one native FP64 complex multiply-add.
//
// Algorithms (all published error-free transformations and double-word
// operations):
//   TwoSum            Knuth, TAOCP vol. 2, Sec. 4.2.2 (Theorem B): s + e = a + b exactly.
//   FastTwoSum        Dekker 1971: the same when |a| >= |b|.
//   TwoProd           with an FMA: p + e = a * b exactly.
//   add               Joldes, Muller, Popescu, "Tight and rigorous error bounds
//                     for basic building blocks of double-word arithmetic"
//                     (ACM TOMS 2017), Algorithm 6 (relative error <= 3u^2).
//   sloppy add        same paper, Algorithm 5: absolute error <= ~u^2 (|x| + |y|),
//                     the error model of an adder without a guard digit, under
//                     which the backward error analyses of dot products,
//                     Householder reflections and Jacobi rotations still hold
//                     (Higham, "Accuracy and Stability of Numerical Algorithms",
//                     Sec. 2.4); used inside fma, i.e. for the accumulations.
//   mul               same paper, Algorithm 12 (relative error <= 5u^2).
//   div, sqrt         one Newton / Dekker correction of the FP32 quotient or
//                     root, computed with TwoProd residuals.
// u = 2^-24, so every operation is accurate to a few units of 2^-48.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define TJM_HD __host__ __device__ __forceinline__
#else
#define TJM_HD inline
#endif

namespace tjm {

// The df64 overloads of sqrt, fabs and fma below would otherwise hide the
// global float / double ones for every unqualified call inside namespace tjm.
using ::fabs;
using ::fma;
using ::sqrt;

struct df64 {
  float hi, lo;
  TJM_HD df64() : hi(0.f), lo(0.f) {}
  TJM_HD df64(float h, float l) : hi(h), lo(l) {}
  // every conversion into df64 is explicit, so no float or double expression
  // is ever promoted to double-float arithmetic by accident
  TJM_HD explicit df64(float x) : hi(x), lo(0.f) {}
  TJM_HD explicit df64(int x) : hi((float)x), lo(0.f) {}
  // exact split of a double into the nearest FP32 and the FP32 nearest to the rest
  TJM_HD explicit df64(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  TJM_HD explicit operator double() const { return (double)hi + (double)lo; }
  TJM_HD explicit operator float() const { return hi + lo; }
};

TJM_HD df64 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df64(s, e);
}
TJM_HD df64 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}
TJM_HD df64 df_two_prod(float a, float b) {
  const float p = a * b;
  return df64(p, fmaf(a, b, -p));
}

// accurate addition (relative error <= 3u^2)
TJM_HD df64 operator+(df64 x, df64 y) {
  const df64 s = df_two_sum(x.hi, y.hi);
  const df64 t = df_two_sum(x.lo, y.lo);
  const df64 v = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(v.hi, t.lo + v.lo);
}
TJM_HD df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
TJM_HD df64 operator-(df64 x, df64 y) { return x + (-y); }
// sloppy addition: backward error <= ~u^2 on each operand
TJM_HD df64 df_add_sloppy(df64 x, df64 y) {
  const df64 s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
TJM_HD df64 operator*(df64 x, df64 y) {
  const df64 c = df_two_prod(x.hi, y.hi);
  const float t = fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, x.lo * y.lo));
  return df_fast_two_sum(c.hi, c.lo + t);
}
TJM_HD df64 operator/(df64 x, df64 y) {
  // q1 = x / y in FP32, r = x - q1 y exactly enough in double-word, q2 = r / y
  const float q1 = x.hi / y.hi;
  const df64 p = df_two_prod(q1, y.hi);
  const float r = ((x.hi - p.hi) - p.lo + x.lo) - q1 * y.lo;
  const float q2 = r / y.hi;
  return df_fast_two_sum(q1, q2);
}
TJM_HD df64 sqrt(df64 a) {
  if (!(a.hi > 0.f)) return df64(a.hi == 0.f ? 0.f : sqrtf(a.hi), 0.f);
  const float s = sqrtf(a.hi);
  const df64 p = df_two_prod(s, s);
  const float r = ((a.hi - p.hi) - p.lo + a.lo) / (2.f * s);
  return df_fast_two_sum(s, r);
}
TJM_HD df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
// a * b + c with the accumulation done by the sloppy adder
TJM_HD df64 fma(df64 a, df64 b, df64 c) { return df_add_sloppy(a * b, c); }

// a b + c d and acc + a b + c d with a single renormalisation: both products
// split exactly (TwoProd on the high words), their sum and the accumulator
// added by TwoSum, all low-order terms gathered in one FP32 word.  Error
// bounded like the sloppy adder's (a few u^2 of |a b| + |c d| + |acc|); the
// building block of the complex multiply-adds and Jacobi rotations below.
TJM_HD df64 df_dot2(df64 a, df64 b, df64 c, df64 d) {
  const float p = a.hi * b.hi, q = c.hi * d.hi;
  const float ep = fmaf(a.hi, b.hi, -p), eq = fmaf(c.hi, d.hi, -q);
  const df64 s = df_two_sum(p, q);
  float t = s.lo + (ep + eq);
  t = fmaf(a.hi, b.lo, t);
  t = fmaf(a.lo, b.hi, t);
  t = fmaf(c.hi, d.lo, t);
  t = fmaf(c.lo, d.hi, t);
  return df_fast_two_sum(s.hi, t);
}
TJM_HD df64 df_fma2(df64 acc, df64 a, df64 b, df64 c, df64 d) {
  const float p = a.hi * b.hi, q = c.hi * d.hi;
  const float ep = fmaf(a.hi, b.hi, -p), eq = fmaf(c.hi, d.hi, -q);
  const df64 s = df_two_sum(p, q);
  const df64 u = df_two_sum(acc.hi, s.hi);
  float t = u.lo + s.lo + (ep + eq) + acc.lo;
  t = fmaf(a.hi, b.lo, t);
  t = fmaf(a.lo, b.hi, t);
  t = fmaf(c.hi, d.lo, t);
  t = fmaf(c.lo, d.hi, t);
  return df_fast_two_sum(u.hi, t);
}

TJM_HD df64& operator+=(df64& x, df64 y) { x = df_add_sloppy(x, y); return x; }
TJM_HD df64& operator-=(df64& x, df64 y) { x = df_add_sloppy(x, -y); return x; }
TJM_HD df64& operator*=(df64& x, df64 y) { x = x * y; return x; }

// comparisons on the value hi + lo (normalised: hi decides unless equal)
TJM_HD bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
TJM_HD bool operator>(df64 a, df64 b) { return b < a; }
TJM_HD bool operator<=(df64 a, df64 b) { return !(b < a); }
TJM_HD bool operator>=(df64 a, df64 b) { return !(a < b); }
TJM_HD bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
TJM_HD bool operator!=(df64 a, df64 b) { return !(a == b); }

#if defined(__CUDACC__)
__device__ __forceinline__ df64 shfl_xor_df(unsigned m, df64 v, int o) {
  return df64(__shfl_xor_sync(m, v.hi, o), __shfl_xor_sync(m, v.lo, o));
}
#endif

}  // namespace tjm

#undef TJM_HD
