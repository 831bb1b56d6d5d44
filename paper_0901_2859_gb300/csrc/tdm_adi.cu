// tdm_adi.cu -- the right-hand side of one Peaceman-Rachford half step
// (Section 4b, eqs. adi_iter, adi_iter2) in one pass.
//
// A half step solves, along axis a for every line b of every problem s,
//   tridiag(-1, 2 + omega h^2, -1) w = h^2 (omega v + Lambda_b v + f),
// and scaled by h^2 its right-hand side is
//   r[a][b][s] = (omega h^2 - 2) v[a][b][s] + h^2 f[a][b][s] + v[a][b-1][s] + v[a][b+1][s]
// with v = 0 beyond b's ends.  The solver takes it as the rows a of a series
// whose columns are (b, s).  The second half step of an iteration runs along
// the other axis, so v and f arrive as transposed views: element (a, b, s) at
// a * sa + b * sb + s.  Both layouts keep s contiguous.  A thread takes one
// (a, s) and kRhsB consecutive lines b, holding v of lines b0 - 1 .. b0 + kRhsB
// in registers (the window each line's neighbours come from); the lanes of a
// warp take consecutive s, so every load and store of a line is one contiguous
// run.  The pass reads v and f once (the window's two extra lines come from
// cache) and writes r once, in the solver's precision, with no transpose buffer.
//
// Arithmetic.  For smooth v the sum cancels: |r| is about omega h^2 |v|, far
// below |v|, and the solve multiplies an error in r by up to 1 / (omega h^2).
// So a binary64 v needs the sum to about 2^-45 |v|, and binary64 arithmetic
// runs at a small fraction of the binary32 rate on this part.  Binary64 inputs
// are therefore split into pairs of binary32 numbers by integer operations on
// their encodings (truncated high part, the remaining 29 bits rounded into the
// low part: 2^-47 relative), and the sum is formed in pair arithmetic
// (Dekker's exact sum and product, Knuth's two-sum) on the binary32 pipes.
// Each binary64 value is split once.  A thread whose window holds a value
// outside the pairs' range (|x| below 2^-74 or at 2^128 and above, but not 0,
// and non-finite values) loads them again and forms its lines in binary64, and
// every thread does when c or h^2 is nonzero and outside [2^-60, 2^60].  A
// binary64 result is formed in binary64; binary32 inputs are summed in
// binary32, the precision their state already has.
#include <stdint.h>

#include "tdm_internal.cuh"

namespace {

constexpr int kRhsThreads = 256;
constexpr int kRhsB = 4;   // lines b per thread: 4 with 64 registers (4 CTAs per SM) measured fastest

struct Pair {
  float h, l;
};

// x as h + l, h the binary64 value truncated to 24 bits, l the remaining 29
// bits rounded to 24; ok = false where the pair's exponents leave the binary32
// normal range.  0 and binary64 subnormals give (0, 0).
__device__ __forceinline__ Pair split64(double x, bool& ok) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e == 0) return Pair{0.0f, 0.0f};
  if (e < 949u || e > 1150u) {
    ok = false;
    return Pair{0.0f, 0.0f};
  }
  const unsigned sign = hi & 0x80000000u;
  const float h = __uint_as_float(sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  // the low 29 bits weigh 2^(e - 1075); 2^(e - 1075) has the binary32 exponent field e - 948
  const float l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((e - 948u) << 23));
  return Pair{h, sign ? -l : l};
}

// Knuth's two-sum on the high parts, the low parts added into the error, renormalized
__device__ __forceinline__ Pair pair_add(Pair a, Pair b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return Pair{h, __fsub_rn(e, __fsub_rn(h, s))};
}

// Dekker's product by a fused multiply-add for the exact error of the high parts
__device__ __forceinline__ Pair pair_mul(Pair a, Pair b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return Pair{h, __fsub_rn(e, __fsub_rn(h, p))};
}

// grid: x over (chunk of kRhsB lines, s) of a row, y over rows a
template <typename TI, typename TO>
__global__ void __launch_bounds__(kRhsThreads, 4) k_adi_rhs(const TI* __restrict__ v, int64_t va, int64_t vb,
                                                         const TI* __restrict__ f, int64_t fa, int64_t fb,
                                                         int64_t na, unsigned nb, unsigned S, unsigned nchunks,
                                                         double c, double h2, Pair cp, Pair hp, bool pairs,
                                                         TO* __restrict__ r, int64_t ldr) {
  const unsigned t = blockIdx.x * kRhsThreads + threadIdx.x;
  if (t >= S * nchunks) return;   // no barrier below
  const unsigned chunk = t / S, s = t - chunk * S;
  const int64_t b0 = (int64_t)chunk * kRhsB;
  for (int64_t a = blockIdx.y; a < na; a += gridDim.y) {
    const TI* vp = v + a * va + s;
    const TI* fp = f + a * fa + s;
    TO* rp = r + a * ldr + s;
    auto ldv = [&](int k) -> TI {   // v of line b0 + k - 1, 0 beyond the ends
      const int64_t bb = b0 + k - 1;
      return (bb >= 0 && bb < (int64_t)nb) ? vp[bb * vb] : TI(0);
    };
    auto ldf = [&](int k) -> TI { return b0 + k < (int64_t)nb ? fp[(b0 + k) * fb] : TI(0); };
    if constexpr (sizeof(TI) == 8 && sizeof(TO) == 4) {
      // split as loaded (the raw values are not kept: a window that needs the
      // binary64 path loads them again)
      bool ok = pairs;
      Pair pw[kRhsB + 2], pf[kRhsB];
#pragma unroll
      for (int k = 0; k < kRhsB + 2; ++k) pw[k] = split64(ldv(k), ok);
#pragma unroll
      for (int k = 0; k < kRhsB; ++k) pf[k] = split64(ldf(k), ok);
      if (ok) {
#pragma unroll
        for (int k = 0; k < kRhsB; ++k) {
          if (b0 + k >= (int64_t)nb) break;
          const Pair q = pair_add(pair_add(pair_add(pw[k], pw[k + 2]), pair_mul(cp, pw[k + 1])), pair_mul(hp, pf[k]));
          rp[(b0 + k) * S] = __fadd_rn(q.h, q.l);
        }
        continue;
      }
    }
    TI w[kRhsB + 2], y[kRhsB];
#pragma unroll
    for (int k = 0; k < kRhsB + 2; ++k) w[k] = ldv(k);
#pragma unroll
    for (int k = 0; k < kRhsB; ++k) y[k] = ldf(k);
#pragma unroll
    for (int k = 0; k < kRhsB; ++k) {
      if (b0 + k >= (int64_t)nb) break;
      if constexpr (sizeof(TI) == 8)
        rp[(b0 + k) * S] = (TO)(c * w[k + 1] + h2 * y[k] + w[k] + w[k + 2]);
      else
        rp[(b0 + k) * S] = (TO)((float)c * w[k + 1] + (float)h2 * y[k] + w[k] + w[k + 2]);
    }
  }
}

Pair host_pair(double x) {
  const float h = (float)x;
  return Pair{h, (float)(x - (double)h)};
}

// c and h^2 as pairs keep 2^-47 only well inside the binary32 range
bool pair_range(double x) {
  const double ax = x < 0 ? -x : x;
  return ax == 0.0 || (ax >= 0x1p-60 && ax <= 0x1p60);
}

}  // namespace

extern "C" tdm_status tdm_adi_rhs(const void* v, int64_t va, int64_t vb, const void* f, int64_t fa, int64_t fb,
                                  int64_t na, int64_t nb, int64_t S, double c, double h2, int in_f64, void* R,
                                  int64_t ldR, int out_f64, void* stream) {
  if (na < 0 || nb < 0 || S < 0 || (!in_f64 && out_f64)) return TDM_ERR_INVALID_ARG;
  if (na == 0 || nb == 0 || S == 0) return TDM_OK;
  if (!v || !f || !R || ldR < nb * S || nb * S > (int64_t)INT32_MAX) return TDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  const unsigned nchunks = (unsigned)((nb + kRhsB - 1) / kRhsB);
  const dim3 grid((unsigned)(((int64_t)nchunks * S + kRhsThreads - 1) / kRhsThreads), (unsigned)(na < 65535 ? na : 65535));
  const Pair cp = host_pair(c), hp = host_pair(h2);
  const bool pairs = pair_range(c) && pair_range(h2);
  if (in_f64 && out_f64)
    k_adi_rhs<double, double><<<grid, kRhsThreads, 0, s>>>(static_cast<const double*>(v), va, vb, static_cast<const double*>(f),
                                                   fa, fb, na, (unsigned)nb, (unsigned)S, nchunks, c, h2, cp, hp, pairs, static_cast<double*>(R), ldR);
  else if (in_f64)
    k_adi_rhs<double, float><<<grid, kRhsThreads, 0, s>>>(static_cast<const double*>(v), va, vb, static_cast<const double*>(f),
                                                  fa, fb, na, (unsigned)nb, (unsigned)S, nchunks, c, h2, cp, hp, pairs, static_cast<float*>(R), ldR);
  else
    k_adi_rhs<float, float><<<grid, kRhsThreads, 0, s>>>(static_cast<const float*>(v), va, vb, static_cast<const float*>(f),
                                                 fa, fb, na, (unsigned)nb, (unsigned)S, nchunks, c, h2, cp, hp, pairs, static_cast<float*>(R), ldR);
  return cudaGetLastError() == cudaSuccess ? TDM_OK : TDM_ERR_CUDA;
}
