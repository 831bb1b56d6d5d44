// tdm_refine.cu -- binary32 dichotomy solves with iterative refinement: F in
// binary32, X in binary64, accuracy of a binary64 solve (or better); one
// persistent kernel that serves a single series (tdm_solve) and many series of
// different sizes (tdm_solve_batched).
//
// Work items.  An item is one tile of R right-hand sides of one series
// A X = F.  A thread-block cluster processes one item at a time with all n rows
// (CTA c owns m blocks of t rows, thread (block, rhs) owns one block for one
// right-hand side) and walks a list of items.  Per item:
//
//   x   = solve(F)          binary32 sweeps and beta sums (Lemma 1, eq.
//                           beta_symn), separator values by Theorem 2 in
//                           binary32 pairs, and the block interiors
//                           x = y + phiL x(p_b) + phiR x(p_{b+1}) formed with
//                           phi and the separator values as pairs: x is kept
//                           as a pair (xh, xl) carrying no binary32 rounding
//   r   = F - A x           error-free binary32 transformations (below)
//   d   = solve(r)          all binary32 (separator values too)
//   X   = xh + xl + d       rounded once to binary64
//
// One correction is enough at condition numbers of several million: the first
// solve's error is then its smooth part alone (~4e-7 of max|x| at kappa ~ 4e6,
// from the binary32 beta sums), and the correction solve recovers that to its
// own relative accuracy.  Had x been rounded to binary32, the residual would be
// dominated by that rounding (~2^-24 |A| |x|, a rough vector) and the
// correction, whose beta sums see the rough part through binary32 inverse rows,
// would stall near 1e-10.  More corrections (refine_steps > 1, the per-tile
// test, the prepare-time calibration) repeat the residual and the correction.
//
// Rows of a block are held as pairs (row j, row j + t/2) in float2 registers:
// the two halves of a block run through the beta sums, the residual, the
// corrections and the output in lockstep on paired binary32 instructions
// (tdm_f2.cuh); only the sweeps' recurrences walk the rows one at a time.
//
// The residual is formed in row-sum form.  With sigma_i = b_i + a_{i-1} + a_i
// and the fluxes E_i = a_i (x_{i+1} - x_i),
//     (A x)_i = sigma_i x_i - E_{i-1} + E_i,
// so  r_i = F_i - sigma_i x_i + E_{i-1} - E_i.  The differences x_{i+1} - x_i
// are formed exactly from the pair representation and the large terms
// E_{i-1} - E_i cancel exactly in Knuth's TwoSum, so the residual's absolute
// error stays near 2^-48 |E| instead of 2^-24 |A||x|.  No binary64
// instruction is issued per unknown except the final rounding of xh + xl.
// Iterative refinement itself is not part of the paper's method; its
// correction solves are the paper's method in binary32.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "tdm_df.cuh"
#include "tdm_f2.cuh"
#include "tdm_iface_df.cuh"
#include "tdm_kernel_common.cuh"
#include "tdm_refine.cuh"
#include "tdm_tma.cuh"

// Calibration record: for corrections k = 1..kRefineCalibSteps of calibration
// solves, the largest max|d_k| / max|x| over columns and tiles (binary32 bit
// patterns of non-negative values, which order like unsigned integers).
__device__ unsigned g_tdm_calib[kRefineCalibSteps];

namespace {
using namespace tdmk;

// Per-tile test (refine_steps = -1), with ratio_k = max over the tile's columns
// of max|d_k| / max|x|: after the first correction, stop once ratio_1 times the
// plan's contraction (measured at prepare: the size of the second correction
// per unit of the first, which overstates the error left by the first about
// threefold) is below kRefineTol1; after correction k >= 2, once the estimated
// relative error ratio_k^2 / ratio_{k-1} (linear convergence) is below
// kRefineTol.
constexpr float kRefineTol = 1e-12f;
constexpr float kRefineTol1 = 4e-12f;
constexpr int kRefineCap = 4;

// max over columns of (max|d| / max|x|) over the whole cluster; every thread of
// every CTA gets the same value (exact maxima, the same division).  slot holds
// this CTA's per-column maxima [2][R]; one warp per column reads every CTA's
// pair in one round (lanes 0-15: max|d|, lanes 16-31: max|x|).
template <int R>
__device__ __forceinline__ float cluster_ratio(const float* slot, int C, int tid, float* scratch, float* bcast) {
  const int lane = tid & 31, nwarps = blockDim.x >> 5;
  for (int col = tid >> 5; col < R; col += nwarps) {
    const int cc = lane & 15;
    float v = cc < C ? ld_cluster_f32(slot + (lane >> 4) * R + col, (unsigned)cc) : 0.f;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const float mx = __shfl_sync(0xffffffffu, v, 16);
    if (lane == 0) scratch[col] = mx > 0.f ? v / mx : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    float q = 0.f;
    for (int k = 0; k < R; k++) q = fmaxf(q, scratch[k]);
    *bcast = q;
  }
  __syncthreads();
  return *bcast;
}

// per-CTA, per-column maxima of |d| and |x| into slot [2][R]: shuffles over
// the blocks a warp covers, then over the warps
template <int R>
__device__ __forceinline__ void cta_maxima(float md, float mx, float* red, float* slot, int tid) {
  const int lane = tid & 31, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int o = R; o < 32; o <<= 1) {
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane < R) {
    red[(tid >> 5) * R + lane] = md;
    red[(nwarps + (tid >> 5)) * R + lane] = mx;
  }
  __syncthreads();
  if (tid < R) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < nwarps; w++) {
      a = fmaxf(a, red[w * R + tid]);
      b = fmaxf(b, red[(nwarps + w) * R + tid]);
    }
    slot[tid] = a;
    slot[R + tid] = b;
  }
}

// Loads of F and stores of X.  A thread's rows are the rows of its block in
// one column, addressed by 32-bit element offsets from the block's first row
// (the launch requires ld <= kRefMaxLd), each load and store predicated on
// its row's existence (no branch).  Both stream: the data is touched once per
// tile and must not evict the coefficients from L1.
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream_if(const float* p, bool pred) {
  float v;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\tmov.f32 %0, 0f00000000;\n\t"
      "@q ld.global.nc.L1::no_allocate.f32 %0, [%1];\n\t}"
      : "=f"(v) : "l"(p), "r"((int)pred));
  return v;
}
__device__ __forceinline__ void st_stream(double* p, double v) {
  asm volatile("st.global.cs.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void st_stream_if(double* p, double v, bool pred) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.global.cs.f64 [%0], %1;\n\t}"
               ::"l"(p), "d"(v), "r"((int)pred));
}

// Where a thread's rows of F (or X) are and which exist: base = the block's
// first row in the thread's column, ld32 = the row stride, rows = how many of
// the block's rows exist in this column (0 for padding threads).
template <typename T>
struct Rows {
  T* base;
  int ld32;
  int rows;
  __device__ __forceinline__ T* at(int i) const { return base + i * ld32; }
};

// F of rows j and j + t/2, or zeros where the rows do not exist
template <int TT>
__device__ __forceinline__ float2 load_pair(const Rows<const float>& f, int j) {
  constexpr int H = TT / 2;
  return make_float2(ld_stream_if(f.at(j), j < f.rows), ld_stream_if(f.at(j + H), j + H < f.rows));
}
template <int TT>
__device__ __forceinline__ void load_rhs(float2 (&g)[TT / 2], const Rows<const float>& f) {
#pragma unroll
  for (int j = 0; j < TT / 2; j++) g[j] = load_pair<TT>(f, j);
}

// Exact binary32 -> binary64 by rebuilding the bit pattern on the integer
// pipe (the conversion instruction runs at the binary64 rate on GB300), no
// branch: zeros keep their sign, infinities and NaNs stay so.  A subnormal
// input is read as 2^-127 (1 + f) instead of 2^-126 f: only the low word of a
// pair can be one, and then only below 2^-126, under the last bit of any
// solution entry above ~2^-100.
__device__ __forceinline__ double f2d_bits(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t a = u & 0x7fffffffu;
  uint32_t hi = (a >> 3) + 0x38000000u;        // exponent rebiased by 1023 - 127
  hi = a >= 0x7f800000u ? hi + 0x38000000u : hi;   // Inf, NaN: the exponent all ones
  hi = a == 0u ? 0u : hi;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(u << 29));
}
// X = hi + lo rounded once to binary64: hi exactly, lo exactly unless it is
// subnormal (then |lo| < 2^-126, far below the last bit of any hi > 2^-100)
__device__ __forceinline__ double pair_to_f64(float hi, float lo) { return f2d_bits(hi) + f2d_bits(lo); }

// coefficient table reads: shared memory (SM) or the read-only cache
template <bool SM>
__device__ __forceinline__ float tld1(const float* p) {
  if constexpr (SM) return *p;
  else return __ldg(p);
}
template <bool SM>
__device__ __forceinline__ float2 tld2(const float* p) {
  if constexpr (SM) return *reinterpret_cast<const float2*>(p);
  else return __ldg(reinterpret_cast<const float2*>(p));
}
template <bool SM>
__device__ __forceinline__ float4 tld4(const float* p) {
  if constexpr (SM) return *reinterpret_cast<const float4*>(p);
  else return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// this thread's low words of x: a float2 {row j, row j + t/2} per j
__device__ __forceinline__ float2 ldxl(const float* xlp, int j) { return reinterpret_cast<const float2*>(xlp)[j]; }
__device__ __forceinline__ void stxl(float* xlp, int j, float2 v) { reinterpret_cast<float2*>(xlp)[j] = v; }

// row i of the block in the pair registers
template <int H>
__device__ __forceinline__ float& at(float2 (&g)[H], int i) {
  return i < H ? g[i].x : g[i - H].y;
}

// A2 + A3: the beta sums over the block (paired rows), then the forward
// elimination of the local sweep, row by row (g replaced by its result)
template <int TT, bool SM>
__device__ __forceinline__ void forward_pass(float2 (&g)[TT / 2], const float* cb, float& bR, float& bL) {
  constexpr int H = TT / 2;
  float2 sR = make_float2(0.f, 0.f), sL = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < H; j++) {
    const float4 w = tld4<SM>(cb + j * kRefTP + kRT_GR);
    sR = f2fma(lo2(w), g[j], sR);
    sL = f2fma(hi2(w), g[j], sL);
  }
  bR = sR.x + sR.y;
  bL = sL.x + sL.y;
  float e = 0.f;
#pragma unroll
  for (int i = 0; i < TT; i += 4) {
    const float4 lf = tld4<SM>(cb + kRefLF(TT) + i);
    e = fmaf(-lf.x, e, at<H>(g, i));
    at<H>(g, i) = e;
    e = fmaf(-lf.y, e, at<H>(g, i + 1));
    at<H>(g, i + 1) = e;
    e = fmaf(-lf.z, e, at<H>(g, i + 2));
    at<H>(g, i + 2) = e;
    e = fmaf(-lf.w, e, at<H>(g, i + 3));
    at<H>(g, i + 3) = e;
  }
}

// A5, first part: the back substitution of the local sweep (independent of the
// separator values), y replaces g
template <int TT, bool SM>
__device__ __forceinline__ void backward_y(float2 (&g)[TT / 2], const float* cb) {
  constexpr int H = TT / 2;
  float y = 0.f;
#pragma unroll
  for (int w = 0; w < TT; w += 2) {   // rows TT-1-w and TT-2-w
    const float4 ci = tld4<SM>(cb + kRefCI(TT) + 2 * w);   // (off-diagonal, 1 / pivot) of both rows
    y = fmaf(-ci.x, y, at<H>(g, TT - 1 - w)) * ci.y;
    at<H>(g, TT - 1 - w) = y;
    y = fmaf(-ci.z, y, at<H>(g, TT - 2 - w)) * ci.w;
    at<H>(g, TT - 2 - w) = y;
  }
}

// A5 of the first solve, as pairs: x = y + phiL xL + phiR xR with phi = PH + PL
// and the separator values xL, xR pairs; the two products are exact up to
// their cross terms and the three-term sum is carried exactly, so x = (xh, xl)
// is the binary32 local solution plus the correction to ~2^-48.  The loads of
// F for the residual are issued as each row pair frees its registers.
template <int TT, bool SM>
__device__ __forceinline__ void first_correction(float2 (&g)[TT / 2], float2 (&xh)[TT / 2], float* xlp, const float* cb,
                                                 f2pair xL, f2pair xR, const Rows<const float>& f, float& maxx) {
  constexpr int H = TT / 2;
  const float2 xLh = f2dup(xL.h), xLl = f2dup(xL.l), xRh = f2dup(xR.h), xRl = f2dup(xR.l);
  const float2 nxLh = f2dup(-xL.h), nxRh = f2dup(-xR.h);
#pragma unroll
  for (int j = 0; j < H; j++) {
    const float4 ph = tld4<SM>(cb + j * kRefTP + kRT_PLH);   // PLH pair, PRH pair
    const float4 pl = tld4<SM>(cb + j * kRefTP + kRT_PLL);   // PLL pair, PRL pair
    // products and their exact errors (the negated products give the errors'
    // addends without a negation)
    const float2 pL = f2mul(lo2(ph), xLh);
    float2 eL = f2fma(lo2(ph), xLh, f2mul(lo2(ph), nxLh));
    eL = f2fma(lo2(ph), xLl, eL);
    eL = f2fma(lo2(pl), xLh, eL);
    const float2 pR = f2mul(hi2(ph), xRh);
    float2 eR = f2fma(hi2(ph), xRh, f2mul(hi2(ph), nxRh));
    eR = f2fma(hi2(ph), xRl, eR);
    eR = f2fma(hi2(pl), xRh, eR);
    const df2 s1 = two_sum2(pL, pR);
    const df2 s2 = two_sum2(s1.h, g[j]);
    xh[j] = s2.h;
    stxl(xlp, j, f2add(f2add(eL, eR), f2add(s1.l, s2.l)));
    maxx = fmaxf(maxx, fmaxf(fabsf(s2.h.x), fabsf(s2.h.y)));
    g[j] = load_pair<TT>(f, j);
  }
}

// one residual row pair: r = F - S + Ep - E, with the large fluxes Ep, E
// cancelling exactly in the first TwoSum
__device__ __forceinline__ float2 residual_pair(float2 F, df2 Ep, df2 E, df2 S) {
  const df2 w = two_diff2(Ep.h, E.h);
  const df2 u = two_sum2(F, w.h);
  const df2 v = two_diff2(u.h, S.h);
  const float2 small = f2add(f2sub(f2sub(Ep.l, E.l), S.l), f2add(f2add(w.l, u.l), v.l));
  return f2add(v.h, small);
}

// Residual, first part: the row pairs j = 1 .. H-2 (rows 1 .. H-2 and
// H+1 .. t-2), which need no value from outside the block.  Returns the flux
// pairs E0 = {E_0, E_H} and Elast = {E_{H-2}, E_{t-2}} for the second part.
// g holds F on entry and r on exit.
template <int TT, bool SM>
__device__ __forceinline__ void residual_interior(float2 (&g)[TT / 2], const float2 (&xh)[TT / 2], const float* xlp,
                                                  const float* cb, df2& E0, df2& Elast) {
  constexpr int H = TT / 2;
  df2 X{xh[0], ldxl(xlp, 0)};
  df2 Ep{};
#pragma unroll
  for (int j = 0; j < H - 1; j++) {
    const df2 Xn{xh[j + 1], ldxl(xlp, j + 1)};
    const float4 av = tld4<SM>(cb + j * kRefTP + kRT_A0);   // A0 pair, A1 pair
    const df2 E = df2_mul(df2{lo2(av), hi2(av)}, df2_diff(Xn, X));
    if (j == 0) {
      E0 = E;
    } else {
      const float4 sv = tld4<SM>(cb + j * kRefTP + kRT_S0);   // S0 pair, S1 pair
      const df2 S = df2_mul(df2{lo2(sv), hi2(sv)}, X);
      g[j] = residual_pair(g[j], Ep, E, S);
    }
    Ep = E;
    X = Xn;
  }
  Elast = Ep;
}

// Residual, second part: the row pairs 0 and H-1, with x at the rows just
// outside the block (xm before it, xp after it)
template <int TT, bool SM>
__device__ __forceinline__ void residual_edges(float2 (&g)[TT / 2], const float2 (&xh)[TT / 2], const float* xlp,
                                               const float* cb, f2pair xm, f2pair xp, df2 E0, df2 Elast) {
  constexpr int H = TT / 2;
  const float2 xl0 = ldxl(xlp, 0);
  {   // pair H-1: {E_{H-1}, E_{t-1}} needs x_H (second half's first row) and x_t (outside)
    const df2 X{xh[H - 1], ldxl(xlp, H - 1)};
    const df2 Xn{make_float2(xh[0].y, xp.h), make_float2(xl0.y, xp.l)};
    const float4 av = tld4<SM>(cb + (H - 1) * kRefTP + kRT_A0);
    const df2 E = df2_mul(df2{lo2(av), hi2(av)}, df2_diff(Xn, X));
    const float4 sv = tld4<SM>(cb + (H - 1) * kRefTP + kRT_S0);
    const df2 S = df2_mul(df2{lo2(sv), hi2(sv)}, X);
    g[H - 1] = residual_pair(g[H - 1], Elast, E, S);
    Elast = E;   // now {E_{H-1}, E_{t-1}}
  }
  {   // pair 0: Ep = {E_{-1}, E_{H-1}}, E = E0
    const float2 ap = tld2<SM>(cb + kRefTail(TT));   // a of the row before the block
    const f2pair Em1 = df_mul(f2pair{ap.x, ap.y}, df_diff(f2pair{xh[0].x, xl0.x}, xm));
    const df2 Ep{make_float2(Em1.h, Elast.h.x), make_float2(Em1.l, Elast.l.x)};
    const float4 sv = tld4<SM>(cb + kRT_S0);
    const df2 S = df2_mul(df2{lo2(sv), hi2(sv)}, df2{xh[0], xl0});
    g[0] = residual_pair(g[0], Ep, E0, S);
  }
}

// A5 of a correction solve: d = y + PH_L xL + PH_R xR (binary32), added to x
// with an exact TwoSum (its error joins xl).  maxd = max |d| (for the tests).
// With NEXT, F is reloaded into g for the next residual.
template <int TT, bool SM, bool NEXT>
__device__ __forceinline__ void correction_update(float2 (&g)[TT / 2], float2 (&xh)[TT / 2], float* xlp, const float* cb,
                                                  float xL, float xR, float& maxd, const Rows<const float>& f) {
  constexpr int H = TT / 2;
  const float2 xL2 = f2dup(xL), xR2 = f2dup(xR);
#pragma unroll
  for (int j = 0; j < H; j++) {
    const float4 ph = tld4<SM>(cb + j * kRefTP + kRT_PLH);
    const float2 d = f2fma(hi2(ph), xR2, f2fma(lo2(ph), xL2, g[j]));
    maxd = fmaxf(maxd, fmaxf(fabsf(d.x), fabsf(d.y)));
    const df2 s = two_sum2(xh[j], d);
    xh[j] = s.h;
    stxl(xlp, j, f2add(ldxl(xlp, j), s.l));
    g[j] = NEXT ? load_pair<TT>(f, j) : make_float2(0.f, 0.f);
  }
}

// Output: X = xh + xl (+ d of a last correction not yet added, FUSED) rounded
// once to binary64; then the next item's F into g, row pair by row pair.
template <int TT, bool SM, bool FUSED>
__device__ __forceinline__ void output(float2 (&g)[TT / 2], const float2 (&xh)[TT / 2], const float* xlp, const float* cb,
                                       float xL, float xR, const Rows<double>& x, const Rows<const float>& fn,
                                       float& maxd) {
  constexpr int H = TT / 2;
  const float2 xL2 = f2dup(xL), xR2 = f2dup(xR);
#pragma unroll
  for (int j = 0; j < H; j++) {
    float2 hi = xh[j], lo = ldxl(xlp, j);
    if (FUSED) {
      const float4 ph = tld4<SM>(cb + j * kRefTP + kRT_PLH);
      const float2 d = f2fma(hi2(ph), xR2, f2fma(lo2(ph), xL2, g[j]));
      maxd = fmaxf(maxd, fmaxf(fabsf(d.x), fabsf(d.y)));
      const df2 s = two_sum2(hi, d);
      hi = s.h;
      lo = f2add(lo, s.l);
    }
    st_stream_if(x.at(j), pair_to_f64(hi.x, lo.x), j < x.rows);
    st_stream_if(x.at(j + H), pair_to_f64(hi.y, lo.y), j + H < x.rows);
    g[j] = load_pair<TT>(fn, j);
  }
}

// Shared-memory layout of the refined kernel (byte offsets; the same function
// sizes the launch on the host).
struct RefOffsets {
  size_t tab, xl, edge, red, cvg, ver, iface, bytes;
};
constexpr int kVerSlots = 4;   // rotating slots of speculative tiles' maxima
__host__ __device__ constexpr RefOffsets refine_offsets(int R, int TT, int NT, bool sm_coef) {
  const size_t MM = (size_t)(NT / R);
  RefOffsets o{};
  size_t p = 0;
  o.tab = p; if (sm_coef) p += round16(4 * MM * (size_t)kRefTabStride(TT));
  o.xl = p; p += round16(4 * (size_t)NT * (TT + 2));
  o.edge = p; p += round16(4 * 4 * MM * R);
  o.red = p; p += round16(4 * 2 * (size_t)(NT / 32) * R);
  o.cvg = p; p += round16(4 * 5 * (size_t)R);
  o.ver = p; p += round16(4 * (kVerSlots * 2 + 1) * (size_t)R);
  o.iface = p; p += iface_offsets(R, (int)MM, true).bytes;
  o.bytes = p;
  return o;
}

// Modes of a work item.
//   kFixed   exactly `steps` corrections, the last one added in the output;
//   kSpec    (per-tile test of a calibrated plan) one correction, added in the
//            output at once; the tile's maxima go to a verification slot that
//            the next work item's first interface exchange publishes, and
//            every CTA checks ratio_1 x contraction <= kRefineTol1 there; a
//            tile that fails is solved again, as kRetry, right after;
//   kTested  (per-tile test, uncalibrated) a cluster-wide test after every
//            correction, after the first with the plan's contraction;
//   kRetry   kTested without the first test (one correction was not enough);
//   kCalib   kRefineCalibSteps corrections, every one's size recorded.
enum { kFixed = 0, kSpec = 1, kTested = 2, kRetry = 3, kCalib = 4 };

// ratio_1 of a speculative tile from every CTA's slot (after a cluster barrier
// has published the slots): one warp per column, lanes 0-15 max|d|, 16-31
// max|x|; scratch[col] receives the column's ratio.
template <int R>
__device__ __forceinline__ void verify_columns(const float* slot, int C, float* scratch) {
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int col = threadIdx.x >> 5; col < R; col += nwarps) {
    const int cc = lane & 15;
    float v = cc < C ? ld_cluster_f32(slot + (lane >> 4) * R + col, (unsigned)cc) : 0.f;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const float mx = __shfl_sync(0xffffffffu, v, 16);
    if (lane == 0) scratch[col] = mx > 0.f ? v / mx : 0.f;
  }
}

template <int R, int TT, int NT, int MINB, bool SM>
__global__ void __launch_bounds__(NT, MINB) k_refined(const RefLaunch L) {
  constexpr int H = TT / 2;
  constexpr int MM = NT / R;                               // most blocks a CTA can own
  constexpr int STR = kRefTabStride(TT);
  constexpr int XLS = TT + 2;                              // floats per thread of xl (conflict-free float2 rows)
  constexpr RefOffsets O = refine_offsets(R, TT, NT, SM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float ratio_s;
  float* const stab = reinterpret_cast<float*>(smem_raw + O.tab);    // [MM][STR] coefficient table
  float* const sxl = reinterpret_cast<float*>(smem_raw + O.xl);      // [NT][XLS] low words of x
  float* const eFh = reinterpret_cast<float*>(smem_raw + O.edge);    // [4][MM][R] block edge values of x
  float* const eFl = eFh + MM * R;
  float* const eLh = eFl + MM * R;
  float* const eLl = eLh + MM * R;
  float* const red = reinterpret_cast<float*>(smem_raw + O.red);     // [2][warps][R] per-warp maxima
  float* const cvg = reinterpret_cast<float*>(smem_raw + O.cvg);     // [2][2][R] per-CTA maxima, read remotely
  float* const cvg_scratch = cvg + 4 * R;                            // [R]
  float* const ver = reinterpret_cast<float*>(smem_raw + O.ver);     // [kVerSlots][2][R] speculative tiles' maxima
  float* const ver_scratch = ver + kVerSlots * 2 * R;                // [R]
  const IfaceDF<R, MM, true> f{smem_raw + O.iface};
  const unsigned c = cluster_rank();
  const int tid = threadIdx.x;
  const int r = tid % R;
  const int bl = tid / R;
  const int m = L.m;
  const int cluster_id = blockIdx.x / L.C;
  const int nclusters = gridDim.x / L.C;
  float* const xlp = sxl + tid * XLS;
  // Threads past the CTA's blocks (bl >= m) only round the CTA up to whole
  // warps; they run the same code on zero coefficients and zero data.
  for (int k = tid; k < kVerSlots * 2 * R; k += blockDim.x) ver[k] = 0.f;   // published by the first cluster barrier

#define ITEMX(i, fld) (L.single ? L.one.fld : L.items[i].fld)
  float2 g[H], xh[H];
  int cur_series = -1;
  int parity = 0;
  int preloaded_item = -1;  // the item whose F g holds (loaded during the previous output)
  int next_main = cluster_id;
  int pending = -1;         // a speculative item that failed its verification
  int unverified = -1;      // the last speculative item, its maxima not checked yet
  int vslot = 0;            // and its verification slot
  int nspec = 0;            // speculative items so far (slot rotation)
  while (true) {
    int it;
    bool retry = false;
    if (pending >= 0) {
      it = pending;
      pending = -1;
      retry = true;
    } else if (next_main < L.nitems) {
      it = next_main;
      next_main += nclusters;
    } else if (unverified >= 0) {   // the last speculative item: check it now
      cluster_barrier();
      verify_columns<R>(ver + vslot * 2 * R, L.C, ver_scratch);
      __syncthreads();
      float q = 0.f;
      for (int k = 0; k < R; k++) q = fmaxf(q, ver_scratch[k]);
      if (!(q * ITEMX(unverified, contraction) <= kRefineTol1)) pending = unverified;
      unverified = -1;
      __syncthreads();
      continue;
    } else {
      break;
    }
    // fields of the current item, read where they are used (kernel parameter
    // or work list; no address of the parameter is taken)
#define ITEM(fld) ITEMX(it, fld)
    const int tile = L.single ? it : L.items[it].tile;
    const int M = ITEM(M);
    if (ITEM(series) != cur_series) {   // new series: ratios, products, coefficient rows
      __syncthreads();
      iface_df_setup(f, ITEM(rR), ITEM(rL), M, m, L.C, c);
      if constexpr (SM) {   // this CTA's blocks of the table; blocks past M as zeros
        const float4* src = reinterpret_cast<const float4*>(ITEM(tab) + (size_t)c * m * STR);
        float4* dst = reinterpret_cast<float4*>(stab);
        for (int k = tid; k < MM * STR / 4; k += blockDim.x) {
          const int blk = (k * 4) / STR;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (blk < m && (int)c * m + blk < M) v = __ldg(src + k);
          dst[k] = v;
        }
      }
      __syncthreads();
      cur_series = ITEM(series);
    }
    const int n = ITEM(n);
    const int b = (int)c * m + bl;
    const bool blk_ok = (bl < m) && (b < M);
    const int64_t row0 = (int64_t)b * TT;
    const int nrows = blk_ok ? (int)((n - row0) < TT ? (n - row0) : TT) : 0;
    const int64_t col = (int64_t)tile * R + r;
    const bool col_ok = col < ITEM(N);
    const bool active = nrows > 0 && col_ok;   // this thread's rows and column exist
    const float* cb = SM ? stab + (size_t)bl * STR : ITEM(tab) + (size_t)(blk_ok ? b : M) * STR;
    // this thread's rows of F (none for padding threads and missing columns)
    const Rows<const float> fr{ITEM(F) + row0 * ITEM(ldF) + col, (int)ITEM(ldF), active ? nrows : 0};
    const int steps_cfg = ITEM(steps);
    const int mode = retry ? kRetry
                           : steps_cfg == kRefineCalib ? kCalib
                           : steps_cfg == -1 ? (ITEM(contraction) < 1.f ? kSpec : kTested) : kFixed;
    const bool track = mode == kTested || mode == kRetry || mode == kCalib;
    const int cap = mode == kFixed ? steps_cfg : mode == kSpec ? 1 : mode == kCalib ? kRefineCalibSteps : kRefineCap;

    if (preloaded_item != it) load_rhs<TT>(g, fr);

    // ---- first solve (A2-A5): x = (xh, xl) ------------------------------------
    float maxx = 0.f;
    {
      float bR, bL;
      forward_pass<TT, SM>(g, cb, bR, bL);
      f.beR()[bl * f.kRP + r] = bR;
      f.beL()[bl * f.kRP + r] = bL;
      __syncthreads();
      iface_df_scan<R, MM, true, true>(f, m, parity);
      cluster_arrive();   // the back substitution overlaps the exchange of the CTA totals
      backward_y<TT, SM>(g, cb);
      cluster_wait();
      iface_df_fold<R, MM, true, true>(f, L.C, c, parity);
      // the exchange also published the last speculative tile's maxima
      if (unverified >= 0) verify_columns<R>(ver + vslot * 2 * R, L.C, ver_scratch);
      __syncthreads();
      parity ^= 1;
      if (unverified >= 0) {   // every CTA reaches the same verdict from the same maxima
        float q = 0.f;
        for (int k = 0; k < R; k++) q = fmaxf(q, ver_scratch[k]);
        if (!(q * ITEMX(unverified, contraction) <= kRefineTol1)) pending = unverified;
        unverified = -1;
      }
      f2pair xL{0.f, 0.f}, xR{0.f, 0.f};
      if (blk_ok) {
        if (b >= 1) xL = iface_df_sep_pair<R, MM, true, true>(f, bl, r);
        if (b + 1 <= M - 1) xR = iface_df_sep_pair<R, MM, true, true>(f, bl + 1, r);
      }
      first_correction<TT, SM>(g, xh, xlp, cb, xL, xR, fr, maxx);
    }
    if (!col_ok) maxx = 0.f;

    // ---- corrections: r = F - A x, d = solve(r), x += d ----------------------
    const int64_t ldX = ITEM(ldX);
    const Rows<double> xr{ITEM(X) + row0 * ldX + col, (int)ldX, active ? nrows : 0};
    // the item that runs next, whose F the output loads
    const int nxt = pending >= 0 ? pending : (next_main < L.nitems ? next_main : -1);
    Rows<const float> fn{ITEM(F), 0, 0};
    if (nxt >= 0) {
      const int tile_n = L.single ? nxt : L.items[nxt].tile;
      const int64_t col_n = (int64_t)tile_n * R + r;
      const int n_n = ITEMX(nxt, n);
      if ((bl < m) && (b < ITEMX(nxt, M)) && col_n < ITEMX(nxt, N)) {
        fn.rows = (int)((n_n - row0) < TT ? (n_n - row0) : TT);
        fn.ld32 = (int)ITEMX(nxt, ldF);
        fn.base = ITEMX(nxt, F) + row0 * ITEMX(nxt, ldF) + col_n;
      }
    }
    float ratio_prev = 1.f;
    int done = 0;
    bool fused_out = false;
    while (true) {
      if (done == cap) break;
      // edge values of x for the neighbours' residuals
      eFh[bl * R + r] = xh[0].x;
      eFl[bl * R + r] = ldxl(xlp, 0).x;
      eLh[bl * R + r] = xh[H - 1].y;
      eLl[bl * R + r] = ldxl(xlp, H - 1).y;
      // Tests read every CTA's maxima of the last correction: a full cluster
      // barrier, which also publishes the edge values.  Otherwise the interior
      // of the residual overlaps the edge-value barrier.
      const bool test = track && done >= (mode == kRetry ? 2 : 1);
      if (test) {
        cluster_barrier();
        const float ratio = cluster_ratio<R>(cvg + (done & 1) * 2 * R, L.C, tid, cvg_scratch, &ratio_s);
        if (mode == kCalib && tid == 0 && c == 0) atomicMax(&g_tdm_calib[done - 1], __float_as_uint(ratio));
        if (mode != kCalib) {
          const bool stop = done == 1 ? ratio * ITEM(contraction) <= kRefineTol1
                                      : ratio * ratio <= kRefineTol * ratio_prev;
          if (stop) break;
        }
        ratio_prev = ratio;
      } else {
        if (mode == kRetry && done == 1)   // the ratio test of correction 2 needs ratio_1
          ratio_prev = 0.f;
        cluster_arrive();
      }
      df2 E0, Elast;
      residual_interior<TT, SM>(g, xh, xlp, cb, E0, Elast);
      if (!test) cluster_wait();
      if (mode == kRetry && done == 1)
        ratio_prev = cluster_ratio<R>(cvg + (done & 1) * 2 * R, L.C, tid, cvg_scratch, &ratio_s);
      f2pair xm{0.f, 0.f}, xp{0.f, 0.f};   // x at rows row0-1 and row0+TT
      if (bl > 0) {
        xm = f2pair{eLh[(bl - 1) * R + r], eLl[(bl - 1) * R + r]};
      } else if (c > 0) {
        xm = f2pair{ld_cluster_f32(eLh + (m - 1) * R + r, c - 1), ld_cluster_f32(eLl + (m - 1) * R + r, c - 1)};
      }
      if (bl < m - 1) {
        xp = f2pair{eFh[(bl + 1) * R + r], eFl[(bl + 1) * R + r]};
      } else if ((int)c < L.C - 1) {
        xp = f2pair{ld_cluster_f32(eFh + r, c + 1), ld_cluster_f32(eFl + r, c + 1)};
      }
      residual_edges<TT, SM>(g, xh, xlp, cb, xm, xp, E0, Elast);

      // ---- correction solve, all binary32 --------------------------------------
      float bR, bL;
      forward_pass<TT, SM>(g, cb, bR, bL);
      f.beR()[bl * f.kRP + r] = bR;
      f.beL()[bl * f.kRP + r] = bL;
      __syncthreads();
      iface_df_scan<R, MM, true, false>(f, m, parity);
      cluster_arrive();
      backward_y<TT, SM>(g, cb);
      cluster_wait();
      iface_df_fold<R, MM, true, false>(f, L.C, c, parity);
      __syncthreads();
      parity ^= 1;
      float xL = 0.f, xR = 0.f;
      if (blk_ok) {
        if (b >= 1) xL = iface_df_sep_pair<R, MM, true, false>(f, bl, r).h;
        if (b + 1 <= M - 1) xR = iface_df_sep_pair<R, MM, true, false>(f, bl + 1, r).h;
      }
      done++;
      if (!track && done == cap) {   // the last correction is added in the output
        float maxd = 0.f;
        output<TT, SM, true>(g, xh, xlp, cb, xL, xR, xr, fn, maxd);
        fused_out = true;
        if (mode == kSpec) {   // this CTA's per-column maxima into the tile's verification slot
          const int slot = nspec % kVerSlots;
          if (!col_ok) maxd = 0.f;
          float md = maxd, mx = maxx;
#pragma unroll
          for (int o = R; o < 32; o <<= 1) {
            md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          }
          if ((tid & 31) < R) {
            atomicMax(reinterpret_cast<unsigned*>(ver) + (slot * 2 + 0) * R + r, __float_as_uint(md));
            atomicMax(reinterpret_cast<unsigned*>(ver) + (slot * 2 + 1) * R + r, __float_as_uint(mx));
          }
          // the slot two speculative tiles ahead: its last readers have passed
          // at least one cluster barrier since
          const int z = (nspec + 2) % kVerSlots;
          if (tid < 2 * R) ver[z * 2 * R + tid] = 0.f;
          unverified = it;
          vslot = slot;
          nspec++;
        }
        break;
      }
      float maxd = 0.f;
      if (done < cap) correction_update<TT, SM, true>(g, xh, xlp, cb, xL, xR, maxd, fr);
      else correction_update<TT, SM, false>(g, xh, xlp, cb, xL, xR, maxd, fr);
      if (track) {
        if (!col_ok) maxd = 0.f;   // padding columns of a ragged tile do not vote
        cta_maxima<R>(maxd, maxx, red, cvg + (done & 1) * 2 * R, tid);
      }
    }
    if (!fused_out) {
      if (track && done == cap) {   // cap reached: record the last correction
        cluster_barrier();
        const float ratio = cluster_ratio<R>(cvg + (done & 1) * 2 * R, L.C, tid, cvg_scratch, &ratio_s);
        if (mode == kCalib && tid == 0 && c == 0) atomicMax(&g_tdm_calib[done - 1], __float_as_uint(ratio));
        if (mode != kCalib && tid == 0 && !(ratio * ratio <= kRefineTol * ratio_prev)) atomicExch(L.err, kDevErrNotConverged);
      }
      float unused = 0.f;
      output<TT, SM, false>(g, xh, xlp, cb, 0.f, 0.f, xr, fn, unused);
    }
    preloaded_item = nxt;
#undef ITEM
  }
#undef ITEMX
  // no CTA may leave while a peer can still read its shared memory
  cluster_barrier();
}

template <int R, int TT, int NT, int MINB, bool SM>
tdm_status launch_shape(const RefShape& sh, const RefLaunch& L, int nitems, cudaStream_t s) {
  auto kern = k_refined<R, TT, NT, MINB, SM>;
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t, int>, int> occ;   // (device, C, smem, threads) -> clusters
  int dev = 0;
  cudaGetDevice(&dev);
  TDM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
  if (sh.C > 8) TDM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = sh.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(sh.threads);
  lc.dynamicSmemBytes = sh.smem;
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  int maxc = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(dev, sh.C, sh.smem, sh.threads);
    auto it = occ.find(key);
    if (it != occ.end()) {
      maxc = it->second;
    } else {
      lc.gridDim = dim3(sh.C);
      if (cudaOccupancyMaxActiveClusters(&maxc, (void*)kern, &lc) != cudaSuccess || maxc < 1) {
        (void)cudaGetLastError();
        maxc = 1;
      }
      occ[key] = maxc;
    }
  }
  const int nclusters = nitems < maxc ? nitems : maxc;
  lc.gridDim = dim3(nclusters * sh.C);
  TDM_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, L));
  return TDM_OK;
}

struct RefCand {
  int R, NT;
  bool sm;
};
// the shapes of each block size, in the rule's order
constexpr RefCand kCand32[] = {{8, 256, true}, {8, 512, true}, {4, 512, false}, {16, 512, true}};
constexpr RefCand kCand16[] = {{8, 256, true}, {8, 512, true}, {4, 1024, false}};
constexpr int kRule32 = 3, kRule16 = 3;   // candidates the rule tries (the rest only on request)

}  // namespace

// Tile shapes: R right-hand sides per tile, NT threads per CTA, m = NT / R
// blocks of t rows per CTA, up to 16 CTAs per cluster.
//   t = 32: R = 8, 256 threads, two CTAs per SM, table in shared memory
//           (n <= 16384); R = 8, 512 threads (n <= 32768); R = 4, 512 threads,
//           table read through L1 (n <= 65536); R = 16, 512 threads on request.
//   t = 16: R = 8, 256 threads (n <= 8192); R = 8, 512 threads (n <= 16384);
//           R = 4, 1024 threads, table through L1 (n <= 65536).
// A requested width (pref) is tried first; the rule's shapes follow.
bool tdm_refined_shape(int M, int t, int pref, RefShape& sh) {
  const RefCand* cand = t == 16 ? kCand16 : kCand32;
  const int ncand = t == 16 ? (int)(sizeof(kCand16) / sizeof(kCand16[0])) : (int)(sizeof(kCand32) / sizeof(kCand32[0]));
  const int nrule = t == 16 ? kRule16 : kRule32;
  auto fits = [&](const RefCand& k) -> bool {
    const int m_max = k.NT / k.R;
    const int C = (M + m_max - 1) / m_max;
    if (C > 16) return false;
    const int m = (M + C - 1) / C;
    const size_t smem = refine_offsets(k.R, t, k.NT, k.sm).bytes;
    if (smem > 227 * 1024) return false;
    sh.R = k.R; sh.NT = k.NT; sh.m = m; sh.C = C;
    sh.threads = ((m * k.R + 31) / 32) * 32;
    if (sh.threads < 96) sh.threads = 96;
    sh.sm_coef = k.sm;
    sh.smem = smem;
    return true;
  };
  if (pref)
    for (int k = 0; k < ncand; k++)
      if (cand[k].R == pref && fits(cand[k])) return true;
  for (int k = 0; k < nrule; k++)
    if (fits(cand[k])) return true;
  return false;
}

tdm_status tdm_refined_launch(const RefShape& sh, int t, const RefItem* items, const RefItem* one, int nitems,
                              int* err, cudaStream_t s) {
  if (nitems <= 0) return TDM_OK;
  RefLaunch L;
  memset(&L, 0, sizeof(L));
  L.items = items;
  if (one) L.one = *one;
  L.nitems = nitems;
  L.single = items ? 0 : 1;
  L.m = sh.m;
  L.C = sh.C;
  L.err = err;
  const int key = sh.R * 100000 + sh.NT * 10 + (t == 16 ? 1 : 0);
  switch (key) {
    case 8 * 100000 + 256 * 10 + 0: return launch_shape<8, 32, 256, 2, true>(sh, L, nitems, s);
    case 8 * 100000 + 512 * 10 + 0: return launch_shape<8, 32, 512, 1, true>(sh, L, nitems, s);
    case 4 * 100000 + 512 * 10 + 0: return launch_shape<4, 32, 512, 1, false>(sh, L, nitems, s);
    case 16 * 100000 + 512 * 10 + 0: return launch_shape<16, 32, 512, 1, true>(sh, L, nitems, s);
    case 8 * 100000 + 256 * 10 + 1: return launch_shape<8, 16, 256, 2, true>(sh, L, nitems, s);
    case 8 * 100000 + 512 * 10 + 1: return launch_shape<8, 16, 512, 1, true>(sh, L, nitems, s);
    case 4 * 100000 + 1024 * 10 + 1: return launch_shape<4, 16, 1024, 1, false>(sh, L, nitems, s);
  }
  return TDM_ERR_NOT_IMPLEMENTED;
}

RefItem tdm_refined_item(const tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                         int series) {
  RefItem it;
  memset(&it, 0, sizeof(it));
  it.F = F; it.X = X; it.ldF = ldF; it.ldX = ldX;
  it.tab = p->rtab; it.rR = p->rR; it.rL = p->rL;
  it.n = (int)p->n; it.M = p->M; it.N = (int)N; it.tile = 0;
  it.series = series;
  it.steps = p->refine_steps;
  it.contraction = p->contraction;
  return it;
}

tdm_status tdm_launch_refined(tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                              cudaStream_t s) {
  if (ldF > kRefMaxLd || ldX > kRefMaxLd) return TDM_ERR_NOT_IMPLEMENTED;
  RefShape sh;
  if (!tdm_refined_shape(p->M, p->t, p->tile_rhs, sh)) return TDM_ERR_NOT_IMPLEMENTED;
  const RefItem one = tdm_refined_item(p, F, ldF, X, ldX, N, 0);
  const int ntiles = (int)((N + sh.R - 1) / sh.R);
  return tdm_refined_launch(sh, p->t, nullptr, &one, ntiles, p->dev_err, s);
}

// Clears / reads the calibration record of the current device.
tdm_status tdm_calibration_record(bool clear, float* ratios, cudaStream_t s) {
  unsigned v[kRefineCalibSteps] = {0, 0, 0, 0};
  if (clear) {
    TDM_CUDA_TRY(cudaMemcpyToSymbolAsync(g_tdm_calib, v, sizeof(v), 0, cudaMemcpyHostToDevice, s));
    TDM_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    TDM_CUDA_TRY(cudaMemcpyFromSymbolAsync(v, g_tdm_calib, sizeof(v), 0, cudaMemcpyDeviceToHost, s));
    TDM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < kRefineCalibSteps; k++) memcpy(&ratios[k], &v[k], sizeof(float));
  }
  return TDM_OK;
}
