// tdm_df.cuh -- "double-float" helpers: a value carried as the unevaluated
// sum hi + lo of two binary32 numbers, manipulated with error-free
// transformations (Knuth's TwoSum, Dekker's Fast2Sum, the FMA-based exact
// product; see Joldes, Muller, Popescu, ACM TOMS 44(2), 2017).  Used by the
// refined solve to form residuals F - A x with binary64-class accuracy on the
// binary32 pipes (GB300 issues binary64 at ~1/70 of the binary32 rate).
#pragma once

struct f2pair {
  float h, l;
};

// s + e == a + b exactly
__device__ __forceinline__ f2pair two_sum_f(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return f2pair{s, (a - (s - bb)) + (b - bb)};
}
// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ f2pair fast_two_sum_f(float a, float b) {
  const float s = a + b;
  return f2pair{s, b - (s - a)};
}
// p + e == a * b exactly
__device__ __forceinline__ f2pair two_prod_f(float a, float b) {
  const float p = a * b;
  return f2pair{p, fmaf(a, b, -p)};
}
// (x1 - x0) for pairs, accurate to ~2^-48 relative to the DIFFERENCE (the
// high and the low words are subtracted exactly).  The result is not
// renormalised: lo is below ~2^-23 hi unless the two differences nearly
// cancel, which keeps the value exact to the same bound.
__device__ __forceinline__ f2pair df_diff(f2pair x1, f2pair x0) {
  const f2pair s = two_sum_f(x1.h, -x0.h);
  const f2pair t = two_sum_f(x1.l, -x0.l);
  const f2pair u = two_sum_f(s.h, t.h);
  return f2pair{u.h, u.l + (s.l + t.l)};
}
// a * x for pairs, not renormalised (hi exact product part, lo carries the rest)
__device__ __forceinline__ f2pair df_mul(f2pair a, f2pair x) {
  const float p = a.h * x.h;
  float e = fmaf(a.h, x.h, -p);
  e = fmaf(a.h, x.l, e);
  e = fmaf(a.l, x.h, e);
  return f2pair{p, e};
}
// a * x for a pair a and a binary32 x
__device__ __forceinline__ f2pair df_mul_f(f2pair a, float x) {
  const float p = a.h * x;
  float e = fmaf(a.h, x, -p);
  e = fmaf(a.l, x, e);
  return f2pair{p, e};
}
// x + d for a pair and a binary32 correction, renormalised
__device__ __forceinline__ f2pair df_add_f(f2pair x, float d) {
  const f2pair s = two_sum_f(x.h, d);
  return fast_two_sum_f(s.h, s.l + x.l);
}
