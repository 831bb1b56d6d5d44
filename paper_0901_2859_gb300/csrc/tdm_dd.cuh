// tdm_dd.cuh -- double-double ("double-word") arithmetic for the preparation
// step: a value is the unevaluated sum hi + lo of two binary64 numbers with
// |lo| <= ulp(hi)/2, giving about 106 significant bits.
//
// Written from the published error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum, the FMA-based exact product, and the double-word sum,
// product and quotient algorithms analysed by Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 44(2), 2017).
#pragma once

struct dd {
  double hi, lo;
};

__host__ __device__ __forceinline__ dd dd_make(double x) { return dd{x, 0.0}; }

// s + e = a + b exactly (Knuth)
__host__ __device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  const double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}
// s + e = a + b exactly, requires |a| >= |b| or a == 0 (Dekker)
__host__ __device__ __forceinline__ dd fast_two_sum(double a, double b) {
  const double s = a + b;
  return dd{s, b - (s - a)};
}
// p + e = a * b exactly (fused multiply-add)
__host__ __device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = a * b;
  return dd{p, fma(a, b, -p)};
}
__host__ __device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  const dd t = two_sum(x.lo, y.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}
__host__ __device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
__host__ __device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
__host__ __device__ __forceinline__ dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  const double e = fma(x.hi, y.lo, x.lo * y.hi);
  return fast_two_sum(p.hi, p.lo + e);
}
__host__ __device__ __forceinline__ dd dd_mul_d(dd x, double y) {
  dd p = two_prod(x.hi, y);
  return fast_two_sum(p.hi, fma(x.lo, y, p.lo));
}
// quotient by two correction steps of long division
__host__ __device__ __forceinline__ dd dd_div(dd x, dd y) {
  const double q1 = x.hi / y.hi;
  dd r = dd_sub(x, dd_mul_d(y, q1));
  const double q2 = r.hi / y.hi;
  r = dd_sub(r, dd_mul_d(y, q2));
  const double q3 = r.hi / y.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, dd_make(q3));
}
__host__ __device__ __forceinline__ double dd_to_d(dd x) { return x.hi + x.lo; }
