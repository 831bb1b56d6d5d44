// tdm_f2.cuh -- two binary32 lanes per instruction.  GB300 executes paired
// binary32 additions, multiplications and fused multiply-adds (PTX add / mul /
// fma .f32x2) at the binary32 rate, so a value held as a float2 of two
// independent numbers costs one instruction per operation for both.  The
// refined solve pairs row i of a block with row i + t/2: the two halves of a
// block then go through the residual, the beta sums and the corrections in
// lockstep.
//
// On top of the lane pairs, the error-free transformations of tdm_df.cuh in
// paired form: Knuth's TwoSum, Dekker's Fast2Sum, the FMA-exact product, and
// the pair ("double-float") operations built from them (Joldes, Muller,
// Popescu, ACM TOMS 44(2), 2017).  Every operation rounds to nearest and is
// never contracted: the intrinsics below are exactly one rounding each.
#pragma once

#include <cuda_runtime.h>

namespace tdmk {

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b = fma(b, -1, a): one paired instruction with a single rounding (the
// product by -1 is exact), so exactly the rounded difference
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// -a, exactly, in one paired instruction
__device__ __forceinline__ float2 f2neg(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ float2 f2dup(float v) { return make_float2(v, v); }

// a pair value per lane: hi + lo
struct df2 {
  float2 h, l;
};

// s + e == a + b exactly, per lane
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  const float2 bb = f2sub(s, a);
  const float2 e = f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb));
  return df2{s, e};
}
// s + e == a - b exactly, per lane (TwoSum of a and -b, without the negation)
__device__ __forceinline__ df2 two_diff2(float2 a, float2 b) {
  const float2 s = f2sub(a, b);
  const float2 bb = f2sub(s, a);
  const float2 e = f2sub(f2sub(a, f2sub(s, bb)), f2add(b, bb));
  return df2{s, e};
}
// s + e == a + b exactly when |a| >= |b| in each lane (or a == 0)
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  return df2{s, f2sub(b, f2sub(s, a))};
}
// x1 - x0 for pairs, to ~2^-48 relative to the difference: the high and the
// low words are subtracted exactly and the two differences combined with one
// more TwoSum (not renormalised; lo stays below ~2^-23 hi).
__device__ __forceinline__ df2 df2_diff(df2 x1, df2 x0) {
  const df2 s = two_diff2(x1.h, x0.h);
  const df2 t = two_diff2(x1.l, x0.l);
  const df2 u = two_sum2(s.h, t.h);
  return df2{u.h, f2add(u.l, f2add(s.l, t.l))};
}
// a * x for pairs, not renormalised: hi is the rounded product of the high
// words, lo carries its exact error and the two cross terms
__device__ __forceinline__ df2 df2_mul(df2 a, df2 x) {
  const float2 p = f2mul(a.h, x.h);
  float2 e = f2fma(a.h, x.h, f2neg(p));
  e = f2fma(a.h, x.l, e);
  e = f2fma(a.l, x.h, e);
  return df2{p, e};
}

}  // namespace tdmk
