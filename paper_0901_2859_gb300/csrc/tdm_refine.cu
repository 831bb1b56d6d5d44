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

#include <algorithm>
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

// Scratch block of a CTA of a cooperative launch (floats): the A4 totals
// [2 parity][2 dir][R] pairs, the edge rows of x (first block: high, low;
// last block: high, low) [4][R], the correction maxima [4][kSlot], the
// speculative maxima [kVerSlots][kSlot].
// Slots of per-CTA maxima that the other CTAs of the cluster read: [2][R]
// (max|d| and max|x| of every column), then the size of the CTA's group and
// its item's contraction.
__host__ __device__ constexpr int kSlot(int R) { return 2 * R + 2; }
constexpr int kVerSlots = 4;   // rotating slots of speculative units' maxima
__host__ __device__ constexpr int kScrEdge(int R) { return 8 * R; }
__host__ __device__ constexpr int kScrCvg(int R) { return 12 * R; }
__host__ __device__ constexpr int kScrVer(int R) { return 12 * R + 4 * kSlot(R); }
__host__ __device__ constexpr int kScr(int R) { return (12 * R + (4 + kVerSlots) * kSlot(R) + 31) / 32 * 32; }

// Relative size max|d| / max|x| of every column for each group of CTAs (the
// maxima taken over the group's CTAs), times the group's contraction when
// `scale`: out[col] receives the largest over the groups of the cluster
// (every CTA computes the same value from the same maxima), own[col] (if not
// null) the value of this CTA's group.  Groups are aligned rank ranges of a
// power-of-two size, or a single group of all CTAs from rank 0, so that the
// xor-shuffles below stay inside a group.  One warp per column: lanes 0-15
// read CTA lane's max|d|, lanes 16-31 CTA (lane - 16)'s max|x|; the slots
// must have been published by a cluster barrier.
// Without groups (GROUPED false) every CTA belongs to the one group of all CL
// CTAs and shares the contraction kc0: nothing but the maxima is read.
template <int R, bool GROUPED, class LK>
__device__ __forceinline__ void group_ratios(const float* slot, int CL, unsigned cphys, bool scale, float kc0,
                                             float* out, float* own, const LK& lk) {
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const unsigned cc = lane & 15;
  const bool have = (int)cc < CL;
  int gs = CL;
  float kc = scale ? kc0 : 1.f;
  if constexpr (GROUPED) {
    gs = have ? (int)lk.ld(slot + 2 * R, cc) : 1;
    kc = have && scale ? lk.ld(slot + 2 * R + 1, cc) : 1.f;
  }
  for (int col = threadIdx.x >> 5; col < R; col += nwarps) {
    float v = have ? lk.ld(slot + (lane >> 4) * R + col, cc) : 0.f;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      const float w = __shfl_xor_sync(0xffffffffu, v, o);
      if (o < gs) v = fmaxf(v, w);
    }
    const float mx = __shfl_down_sync(0xffffffffu, v, 16);
    float q = (lane < 16 && mx > 0.f) ? v / mx * kc : 0.f;
    const float mine = __shfl_sync(0xffffffffu, q, (int)cphys);
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) q = fmaxf(q, __shfl_xor_sync(0xffffffffu, q, o));
    if (lane == 0) {
      out[col] = q;
      if (own) own[col] = mine;
    }
  }
}

// per-CTA, per-column maxima of |d| and |x| into slot (layout of kSlot):
// shuffles over the blocks a warp covers, then over the warps
template <int R>
__device__ __forceinline__ void cta_maxima(float md, float mx, float* red, float* slot, int tid, int gs, float kc) {
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
  if (tid == 0) {
    slot[2 * R] = (float)gs;
    slot[2 * R + 1] = kc;
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
__host__ __device__ constexpr RefOffsets refine_offsets(int R, int TT, int NT, bool sm_coef) {
  const size_t MM = (size_t)(NT / R);
  RefOffsets o{};
  size_t p = 0;
  o.tab = p; if (sm_coef) p += round16(4 * MM * (size_t)kRefTabStride(TT));
  o.xl = p; p += round16(4 * (size_t)NT * (TT + 2));
  o.edge = p; p += round16(4 * 4 * MM * R);
  o.red = p; p += round16(4 * 2 * (size_t)(NT / 32) * R);
  o.cvg = p; p += round16(4 * (4 * (size_t)kSlot(R) + 2 * (size_t)R));
  o.ver = p; p += round16(4 * (kVerSlots * (size_t)kSlot(R) + (size_t)R));
  o.iface = p; p += iface_offsets(R, (int)MM, true).bytes;
  o.bytes = p;
  return o;
}

// Modes of a work item.
//   kFixed   exactly `steps` corrections, the last one added in the output;
//   kSpec    (per-tile test of a calibrated plan) one correction, added in the
//            output at once; the tile's maxima go to a verification slot that
//            the next unit's first interface exchange publishes, and every CTA
//            checks ratio_1 x contraction <= kRefineTol1 there for every
//            group; a unit that fails is solved again right after (kRetry, or
//            kRetryFixed in a grouped launch);
//   kTested  (per-tile test, uncalibrated) a cluster-wide test after every
//            correction, after the first with the plan's contraction;
//   kRetry   kTested without the first test (one correction was not enough);
//   kCalib   kRefineCalibSteps corrections, every one's size recorded;
//   kRetryFixed  (grouped launches, whose groups must all pass the same
//            cluster barriers) kRefineCap corrections, every one's maxima
//            kept; at the end, per group, the tested criterion must hold
//            between some two consecutive corrections.
enum { kFixed = 0, kSpec = 1, kTested = 2, kRetry = 3, kCalib = 4, kRetryFixed = 5 };

// Launch modes: one series (its tile i is unit i); a list of items, one per
// unit, every CTA of the cluster on it (items of one cluster width, each with
// its own blocks per CTA); grouped units (an item per CTA); one series in a
// cooperative launch without clusters (groups of C consecutive CTAs take the
// place of clusters, see Link); runs of a cooperative launch (every CTA walks
// its own list of runs, each a range of tiles of one series on a group of
// consecutive CTAs with a barrier counter of its own).
enum { kLaunchSingle = 0, kLaunchList = 1, kLaunchGrouped = 2, kLaunchCoop = 3, kLaunchCoopRuns = 4 };

template <int R, int TT, int NT, int MINB, bool SM, int LM>
__global__ void __launch_bounds__(NT, MINB) k_refined(const RefLaunch L) {
  constexpr int H = TT / 2;
  constexpr int MM = NT / R;                               // most blocks a CTA can own
  constexpr int STR = kRefTabStride(TT);
  constexpr int XLS = TT + 2;                              // floats per thread of xl (conflict-free float2 rows)
  constexpr int SL = kSlot(R);
  constexpr RefOffsets O = refine_offsets(R, TT, NT, SM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RefItem s_item;                                         // the current item (list, grouped)
  float* const stab = reinterpret_cast<float*>(smem_raw + O.tab);    // [MM][STR] coefficient table
  float* const sxl = reinterpret_cast<float*>(smem_raw + O.xl);      // [NT][XLS] low words of x
  float* const eFh = reinterpret_cast<float*>(smem_raw + O.edge);    // [4][MM][R] block edge values of x
  float* const eFl = eFh + MM * R;
  float* const eLh = eFl + MM * R;
  float* const eLl = eLh + MM * R;
  float* const red = reinterpret_cast<float*>(smem_raw + O.red);     // [2][warps][R] per-warp maxima
  constexpr bool runs = LM == kLaunchCoopRuns;
  constexpr bool coop = LM == kLaunchCoop || runs;
  constexpr bool one_series = LM == kLaunchSingle || LM == kLaunchCoop;
  constexpr bool grouped = LM == kLaunchGrouped;
  // what the peers read: shared memory, or this CTA's scratch block (coop)
  float* const scr = coop ? L.scr + (size_t)blockIdx.x * kScr(R) : nullptr;
  float* const cvg = coop ? scr + kScrCvg(R) : reinterpret_cast<float*>(smem_raw + O.cvg);   // [4][SL] maxima of corrections
  float* const cvg_all = reinterpret_cast<float*>(smem_raw + O.cvg) + 4 * SL;               // [R] largest ratio over the groups
  float* const cvg_own = cvg_all + R;                                                        // [R] ratio of this CTA's group
  float* const ver = coop ? scr + kScrVer(R) : reinterpret_cast<float*>(smem_raw + O.ver);   // [kVerSlots][SL] speculative maxima
  float* const ver_all = reinterpret_cast<float*>(smem_raw + O.ver) + kVerSlots * SL;        // [R]
  float* const scr_e = coop ? scr + kScrEdge(R) : nullptr;                                   // [4][R] edge rows of x
  const IfaceDF<R, MM, true> f{smem_raw + O.iface, coop ? reinterpret_cast<float2*>(scr) : nullptr};
  const int tid = threadIdx.x;
  const int r = tid % R;
  const int bl = tid / R;
  int CL = L.C;                                // CTAs per cluster, or per group (coop; runs: per run)
  unsigned cphys = coop ? blockIdx.x % CL : cluster_rank();
  const int cluster_id = blockIdx.x / CL;
  const int nclusters = gridDim.x / CL;
  Link<coop> lk;
  if constexpr (coop) {
    lk.me = blockIdx.x;
    lk.first = (unsigned)(cluster_id * CL);
    lk.stride = kScr(R);
    lk.g = (unsigned)CL;
    lk.ctr = L.ctr + 32 * cluster_id;
    lk.err = L.err;
  }
  float* const xlp = sxl + tid * XLS;
  // Threads past the CTA's blocks (bl >= m) only round the CTA up to whole
  // warps; they run the same code on zero coefficients and zero data.
  for (int k = tid; k < kVerSlots * SL; k += blockDim.x) ver[k] = 0.f;   // published by the first cluster barrier

#define ITEMX(i, fld) (one_series ? L.one.fld : L.items[i].fld)
  // the item this CTA works on in unit u, and the first rank of its group
  int item0 = 0;   // runs: the item of the run's first tile
  auto item_of = [&](int u) -> int { return grouped ? L.units[u * kUnitW + cphys] : runs ? item0 + u : u; };
  auto group_base = [&](int gs) -> unsigned { return grouped ? (cphys & ~(unsigned)(gs - 1)) : 0u; };
  // largest ratio over the groups (every CTA the same) and this CTA's group's
  auto ratios = [&](const float* slot, float& own) -> float {
    group_ratios<R, grouped>(slot, CL, cphys, false, 1.f, cvg_all, cvg_own, lk);
    __syncthreads();
    float q = 0.f, o = 0.f;
    for (int k = 0; k < R; k++) {
      q = fmaxf(q, cvg_all[k]);
      o = fmaxf(o, cvg_own[k]);
    }
    __syncthreads();
    own = o;
    return q;
  };
  // verdict on the last speculative unit (slot published by a cluster barrier)
  auto verified = [&](int vs, float kc0) -> bool {
    group_ratios<R, grouped>(ver + vs * SL, CL, cphys, true, kc0, ver_all, nullptr, lk);
    __syncthreads();
    float q = 0.f;
    for (int k = 0; k < R; k++) q = fmaxf(q, ver_all[k]);
    return q <= kRefineTol1;
  };
  float2 g[H], xh[H];
  int cur_series = -1;
  int cur_c = -1;
  int parity = 0;
  int preloaded = -1;       // the unit whose F g holds (loaded during the previous output)
  int u_next = grouped ? L.ustart[cluster_id] : cluster_id;
  int u_end = grouped ? L.ustart[cluster_id + 1] : L.nitems;
  const int u_step = grouped || runs ? 1 : nclusters;
  int pending = -1;         // a speculative unit that failed its verification
  int unverified = -1;      // the last speculative unit, its maxima not checked yet
  int vslot = 0;            // and its verification slot
  int nspec = 0;            // speculative units so far (slot rotation)
  const int run_end = runs ? L.ustart[blockIdx.x + 1] : 1;
  for (int run_i = runs ? L.ustart[blockIdx.x] : 0; run_i < run_end; run_i++) {
  if constexpr (runs) {   // a new run: its group, its counter, its tiles; the exchange state starts afresh
    const int rid = L.units[run_i];
    const RefRun rn = L.runs[rid];
    item0 = rn.item0;
    CL = rn.g;
    cphys = blockIdx.x - (unsigned)rn.first;
    lk.first = (unsigned)rn.first;
    lk.g = (unsigned)rn.g;
    lk.ctr = L.ctr + 32 * (size_t)rid;
    lk.narr = 0;
    u_next = 0;
    u_end = rn.ntiles;
    parity = 0;
    preloaded = -1;
    pending = -1;
    unverified = -1;
    nspec = 0;
    // the previous run's peers are done with this CTA's slots (closing barrier)
    for (int k = tid; k < kVerSlots * SL; k += blockDim.x) ver[k] = 0.f;
  }
  while (true) {
    int u;
    bool retry = false;
    if (pending >= 0) {
      u = pending;
      pending = -1;
      retry = true;
    } else if (u_next < u_end) {
      u = u_next;
      u_next += u_step;
    } else if (unverified >= 0) {   // the last speculative unit: check it now
      lk.barrier();
      if (!verified(vslot, ITEMX(item_of(unverified), contraction))) pending = unverified;
      unverified = -1;
      __syncthreads();
      continue;
    } else {
      break;
    }
    // fields of the current item, read where they are used: kernel parameters
    // of a single-series launch, else a copy in shared memory (cheap to read
    // again after every barrier instead of held in registers through the tile)
    const int it = item_of(u);
    if constexpr (!one_series) {
      __syncthreads();   // every read of the previous item's copy is done
      if (tid < (int)(sizeof(RefItem) / 4))
        reinterpret_cast<int*>(&s_item)[tid] = __ldg(reinterpret_cast<const int*>(L.items + it) + tid);
      __syncthreads();
    }
#define ITEM(fld) (one_series ? L.one.fld : s_item.fld)
    // pointers and strides read again at every use (from the copy), so that no
    // address is held in registers through the tile
#define ITEMV(fld) (one_series ? L.one.fld : *(volatile decltype(s_item.fld)*)&s_item.fld)
    const int gs = grouped ? ITEM(g) : CL;   // CTAs of the group
    const int m = one_series ? L.m : ITEM(m);   // blocks per CTA
    const unsigned base = group_base(gs);    // the group's first rank
    const unsigned c = cphys - base;         // rank in the group
    const int tile = one_series ? u : ITEM(tile);
    const int M = ITEM(M);
    // new series or new place in the group: ratios, products, coefficient
    // rows (a null item, M = 0, needs none: its threads have no rows)
    if (M > 0 && (ITEM(series) != cur_series || (int)c != cur_c)) {
      __syncthreads();
      iface_df_setup(f, ITEM(rR), ITEM(rL), M, m, gs, c);
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
      cur_c = (int)c;
    }
    const int n = ITEM(n);
    const int b = (int)c * m + bl;
    const bool blk_ok = (bl < m) && (b < M);
    const bool has_left = blk_ok && b >= 1;          // separators p_b, p_{b+1} inside the matrix
    const bool has_right = blk_ok && b + 1 <= M - 1;
    const int64_t row0 = (int64_t)b * TT;
    const int nrows = blk_ok ? (int)((n - row0) < TT ? (n - row0) : TT) : 0;
    const int64_t col = (int64_t)tile * R + r;
    const bool col_ok = col < ITEM(N);
    const bool active = nrows > 0 && col_ok;   // this thread's rows and column exist
    const float* cb = SM ? stab + (size_t)bl * STR : ITEM(tab) + (size_t)(blk_ok ? b : M) * STR;
    // this thread's rows of F (none for padding threads and missing columns)
    auto rows_F = [&]() {
      return Rows<const float>{ITEMV(F) + row0 * ITEMV(ldF) + col, (int)ITEMV(ldF), active ? nrows : 0};
    };
    const int steps_cfg = ITEM(steps);
#define KC ITEM(contraction)
    int mode;
    if (grouped)
      mode = retry ? kRetryFixed : steps_cfg == -1 ? (KC < 1.f ? kSpec : kRetryFixed) : kFixed;
    else
      mode = retry ? kRetry
                   : steps_cfg == kRefineCalib ? kCalib
                   : steps_cfg == -1 ? (KC < 1.f ? kSpec : kTested) : kFixed;
    const bool intest = mode == kTested || mode == kRetry || mode == kCalib;   // tests between corrections
    const bool track = intest || mode == kRetryFixed;                          // corrections' maxima kept
    const int cap = mode == kFixed ? steps_cfg
                  : mode == kSpec ? 1
                  : mode == kCalib ? kRefineCalibSteps : kRefineCap;

    if (preloaded != u) load_rhs<TT>(g, rows_F());

    // ---- first solve (A2-A5): x = (xh, xl) ------------------------------------
    float maxx = 0.f;
    {
      float bR, bL;
      forward_pass<TT, SM>(g, cb, bR, bL);
      f.beR()[bl * f.kRP + r] = bR;
      f.beL()[bl * f.kRP + r] = bL;
      __syncthreads();
      iface_df_scan<R, MM, true, true>(f, m, parity);
      lk.arrive();   // the back substitution overlaps the exchange of the CTA totals
      backward_y<TT, SM>(g, cb);
      lk.wait();
      iface_df_fold<R, MM, true, true>(f, gs, c, parity, base, lk);
      // the exchange also published the last speculative unit's maxima; every
      // CTA reaches the same verdict from the same maxima
      if (unverified >= 0) {
        if (!verified(vslot, ITEMX(item_of(unverified), contraction))) pending = unverified;
        unverified = -1;
      } else {
        __syncthreads();
      }
      parity ^= 1;
      f2pair xL{0.f, 0.f}, xR{0.f, 0.f};
      if (has_left) xL = iface_df_sep_pair<R, MM, true, true>(f, bl, r);
      if (has_right) xR = iface_df_sep_pair<R, MM, true, true>(f, bl + 1, r);
      first_correction<TT, SM>(g, xh, xlp, cb, xL, xR, rows_F(), maxx);
    }
    if (!col_ok) maxx = 0.f;

    // ---- corrections: r = F - A x, d = solve(r), x += d ----------------------
    auto rows_X = [&]() {
      return Rows<double>{ITEMV(X) + row0 * ITEMV(ldX) + col, (int)ITEMV(ldX), active ? nrows : 0};
    };
    // the unit that runs next, whose F (in its own item's rows) the output loads
    const int nu = pending >= 0 ? pending : (u_next < u_end ? u_next : -1);
    auto rows_next = [&]() {
      Rows<const float> fn{ITEMV(F), 0, 0};
      if (nu >= 0) {
        const int itn = item_of(nu);
        const int gn = grouped ? ITEMX(itn, g) : CL, mn = one_series ? L.m : ITEMX(itn, m);
        const int bn = (int)(cphys - group_base(gn)) * mn + bl;
        const int tile_n = one_series ? nu : L.items[itn].tile;
        const int64_t col_n = (int64_t)tile_n * R + r;
        const int64_t row0_n = (int64_t)bn * TT;
        const int n_n = ITEMX(itn, n);
        if (bl < mn && bn < ITEMX(itn, M) && col_n < ITEMX(itn, N)) {
          fn.rows = (int)((n_n - row0_n) < TT ? (n_n - row0_n) : TT);
          fn.ld32 = (int)ITEMX(itn, ldF);
          fn.base = ITEMX(itn, F) + row0_n * ITEMX(itn, ldF) + col_n;
        }
      }
      return fn;
    };
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
      if constexpr (coop) {   // the rows the neighbouring CTAs read
        if (bl == 0) {
          scr_e[r] = xh[0].x;
          scr_e[R + r] = ldxl(xlp, 0).x;
        }
        if (bl == m - 1) {
          scr_e[2 * R + r] = xh[H - 1].y;
          scr_e[3 * R + r] = ldxl(xlp, H - 1).y;
        }
      }
      // Tests read every CTA's maxima of the last correction: a full cluster
      // barrier, which also publishes the edge values.  Otherwise the interior
      // of the residual overlaps the edge-value barrier.
      const bool test = intest && done >= (mode == kRetry ? 2 : 1);
      if (test) {
        lk.barrier();
        float own;
        const float ratio = ratios(cvg + (done & 1) * SL, own);
        if (mode == kCalib && tid == 0 && c == 0) atomicMax(&g_tdm_calib[done - 1], __float_as_uint(ratio));
        if (mode != kCalib) {
          const bool stop = done == 1 ? ratio * KC <= kRefineTol1 : ratio * ratio <= kRefineTol * ratio_prev;
          if (stop) break;
        }
        ratio_prev = ratio;
      } else {
        if (mode == kRetry && done == 1)   // the ratio test of correction 2 needs ratio_1
          ratio_prev = 0.f;
        lk.arrive();
      }
      df2 E0, Elast;
      residual_interior<TT, SM>(g, xh, xlp, cb, E0, Elast);
      if (!test) lk.wait();
      if (mode == kRetry && done == 1) {
        float own;
        ratio_prev = ratios(cvg + (done & 1) * SL, own);
      }
      f2pair xm{0.f, 0.f}, xp{0.f, 0.f};   // x at rows row0-1 and row0+TT
      if (bl > 0) {
        xm = f2pair{eLh[(bl - 1) * R + r], eLl[(bl - 1) * R + r]};
      } else if (c > 0) {
        if constexpr (coop)
          xm = f2pair{lk.ld(scr_e + 2 * R + r, c - 1), lk.ld(scr_e + 3 * R + r, c - 1)};
        else
          xm = f2pair{ld_cluster_f32(eLh + (m - 1) * R + r, base + c - 1),
                      ld_cluster_f32(eLl + (m - 1) * R + r, base + c - 1)};
      }
      if (bl < m - 1) {
        xp = f2pair{eFh[(bl + 1) * R + r], eFl[(bl + 1) * R + r]};
      } else if ((int)c < gs - 1) {
        if constexpr (coop)
          xp = f2pair{lk.ld(scr_e + r, c + 1), lk.ld(scr_e + R + r, c + 1)};
        else
          xp = f2pair{ld_cluster_f32(eFh + r, base + c + 1), ld_cluster_f32(eFl + r, base + c + 1)};
      }
      residual_edges<TT, SM>(g, xh, xlp, cb, xm, xp, E0, Elast);

      // ---- correction solve, all binary32 --------------------------------------
      float bR, bL;
      forward_pass<TT, SM>(g, cb, bR, bL);
      f.beR()[bl * f.kRP + r] = bR;
      f.beL()[bl * f.kRP + r] = bL;
      __syncthreads();
      iface_df_scan<R, MM, true, false>(f, m, parity);
      lk.arrive();
      backward_y<TT, SM>(g, cb);
      lk.wait();
      iface_df_fold<R, MM, true, false>(f, gs, c, parity, base, lk);
      __syncthreads();
      parity ^= 1;
      float xL = 0.f, xR = 0.f;
      if (has_left) xL = iface_df_sep_pair<R, MM, true, false>(f, bl, r).h;
      if (has_right) xR = iface_df_sep_pair<R, MM, true, false>(f, bl + 1, r).h;
      done++;
      if (!track && done == cap) {   // the last correction is added in the output
        float maxd = 0.f;
        output<TT, SM, true>(g, xh, xlp, cb, xL, xR, rows_X(), rows_next(), maxd);
        fused_out = true;
        if (mode == kSpec) {   // this CTA's per-column maxima into the unit's verification slot
          const int slot = nspec % kVerSlots;
          if (!col_ok) maxd = 0.f;
          float md = maxd, mx = maxx;
#pragma unroll
          for (int o = R; o < 32; o <<= 1) {
            md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          }
          if ((tid & 31) < R) {
            atomicMax(reinterpret_cast<unsigned*>(ver) + slot * SL + r, __float_as_uint(md));
            atomicMax(reinterpret_cast<unsigned*>(ver) + slot * SL + R + r, __float_as_uint(mx));
          }
          if (tid == 0) {
            ver[slot * SL + 2 * R] = (float)gs;
            ver[slot * SL + 2 * R + 1] = KC;
          }
          // the slot two speculative units ahead: its last readers have passed
          // at least one cluster barrier since
          const int z = (nspec + 2) % kVerSlots;
          if (tid < SL) ver[z * SL + tid] = 0.f;
          unverified = u;
          vslot = slot;
          nspec++;
        }
        break;
      }
      float maxd = 0.f;
      if (done < cap) correction_update<TT, SM, true>(g, xh, xlp, cb, xL, xR, maxd, rows_F());
      else correction_update<TT, SM, false>(g, xh, xlp, cb, xL, xR, maxd, rows_F());
      if (track) {   // tested modes alternate two slots; the fixed retry keeps one per correction
        if (!col_ok) maxd = 0.f;   // padding columns of a ragged tile do not vote
        cta_maxima<R>(maxd, maxx, red, cvg + (intest ? (done & 1) : (done - 1) & 3) * SL, tid, gs, KC);
      }
    }
    if (!fused_out) {
      if (track && done == cap) {   // cap reached: record the last correction
        lk.barrier();
        if (mode == kRetryFixed) {   // per group: would the tested criterion have stopped by now?
          float prev, cur;
          ratios(cvg, prev);
          bool conv = false;
          for (int k = 2; k <= cap; k++) {
            ratios(cvg + (k - 1) * SL, cur);
            conv = conv || cur * cur <= kRefineTol * prev;
            prev = cur;
          }
          if (tid == 0 && c == 0 && !conv) atomicExch(L.err, kDevErrNotConverged);
        } else {
          float own;
          const float ratio = ratios(cvg + (done & 1) * SL, own);
          if (mode == kCalib) {
            if (tid == 0 && c == 0) atomicMax(&g_tdm_calib[done - 1], __float_as_uint(ratio));
          } else if (tid == 0 && !(ratio * ratio <= kRefineTol * ratio_prev)) {
            atomicExch(L.err, kDevErrNotConverged);
          }
        }
      }
      float unused = 0.f;
      output<TT, SM, false>(g, xh, xlp, cb, 0.f, 0.f, rows_X(), rows_next(), unused);
    }
    preloaded = nu;
#undef KC
#undef ITEMV
#undef ITEM
  }
  if constexpr (runs) lk.barrier();   // closing: no peer of the run reads this CTA's slots any more
  }
#undef ITEMX
  // no CTA may leave while a peer can still read its shared memory (the
  // scratch blocks of a cooperative launch stay readable)
  if constexpr (!coop) cluster_barrier();
}

template <int R_, int TT_, int NT_, int MINB_, bool SM_>
struct ShapeTag {
  static constexpr int R = R_, TT = TT_, NT = NT_, MINB = MINB_;
  static constexpr bool SM = SM_;
};
// the kernel of a shape: grouped launches, or single-series and list launches
template <class S, int LM>
constexpr auto refined_kernel() { return k_refined<S::R, S::TT, S::NT, S::MINB, S::SM, LM>; }

// launch configuration of a shape's kernel (grid filled in by the caller)
template <class S, int G>
tdm_status shape_config(const RefShape& sh, cudaStream_t s, cudaLaunchConfig_t& lc, cudaLaunchAttribute* at) {
  auto kern = refined_kernel<S, G>();
  TDM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
  if (sh.C > 8) TDM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  lc = cudaLaunchConfig_t{};
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = sh.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(sh.threads);
  lc.dynamicSmemBytes = sh.smem;
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  return TDM_OK;
}

// clusters of the shape that the device holds at once (cached per device,
// cluster size, shared memory and block size)
template <class S, int G>
int shape_max_clusters(const RefShape& sh) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t, int>, int> occ;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_tuple(dev, sh.C, sh.smem, sh.threads);
  auto it = occ.find(key);
  if (it != occ.end()) return it->second;
  cudaLaunchConfig_t lc;
  cudaLaunchAttribute at[1];
  int maxc = 0;
  if (shape_config<S, G>(sh, 0, lc, at) != TDM_OK) maxc = 1;
  lc.gridDim = dim3(sh.C);
  if (maxc == 0 && (cudaOccupancyMaxActiveClusters(&maxc, (void*)refined_kernel<S, G>(), &lc) != cudaSuccess ||
                    maxc < 1)) {
    (void)cudaGetLastError();
    maxc = 1;
  }
  occ[key] = maxc;
  return maxc;
}

template <class S, int G>
tdm_status launch_shape(const RefShape& sh, const RefLaunch& L, int nclusters, cudaStream_t s) {
  cudaLaunchConfig_t lc;
  cudaLaunchAttribute at[1];
  tdm_status st = shape_config<S, G>(sh, s, lc, at);
  if (st != TDM_OK) return st;
  lc.gridDim = dim3(nclusters * sh.C);
  TDM_CUDA_TRY(cudaLaunchKernelEx(&lc, refined_kernel<S, G>(), L));
  return TDM_OK;
}

// calls fn(ShapeTag<...>{}) for the kernel of a shape, false if none
template <class Fn>
bool with_shape(const RefShape& sh, int t, Fn&& fn) {
  const int key = sh.R * 100000 + sh.NT * 10 + (t == 16 ? 1 : 0);
  switch (key) {
    case 8 * 100000 + 256 * 10 + 0: fn(ShapeTag<8, 32, 256, 2, true>{}); return true;
    case 8 * 100000 + 512 * 10 + 0: fn(ShapeTag<8, 32, 512, 1, true>{}); return true;
    case 4 * 100000 + 512 * 10 + 0: fn(ShapeTag<4, 32, 512, 1, false>{}); return true;
    case 16 * 100000 + 512 * 10 + 0: fn(ShapeTag<16, 32, 512, 1, true>{}); return true;
    case 8 * 100000 + 256 * 10 + 1: fn(ShapeTag<8, 16, 256, 2, true>{}); return true;
    case 8 * 100000 + 512 * 10 + 1: fn(ShapeTag<8, 16, 512, 1, true>{}); return true;
    case 4 * 100000 + 1024 * 10 + 1: fn(ShapeTag<4, 16, 1024, 1, false>{}); return true;
  }
  return false;
}

struct RefCand {
  int R, NT;
  bool sm;
};
// A single-series solve runs as a cooperative launch when that holds at least
// kCoopGain times the CTAs that clusters of its width can (clusters of 16 CTAs
// leave a quarter of the GPU's CTA slots idle on GB300, clusters of up to 8
// almost none, and a group barrier in global memory costs more than the
// hardware cluster barrier).
constexpr double kCoopGain = 1.2;
// the shapes of each block size, in the rule's order
constexpr RefCand kCand32[] = {{8, 256, true}, {8, 512, true}, {4, 512, false}, {16, 512, true}};
constexpr RefCand kCand16[] = {{8, 256, true}, {8, 512, true}, {4, 1024, false}};
constexpr int kRule32 = 3, kRule16 = 3;   // candidates the rule tries (the rest only on request)

}  // namespace

// Tile shapes: R right-hand sides per tile, NT threads per CTA, m = NT / R
// blocks of t rows per CTA, up to 16 CTAs per cluster.
//   t = 32: R = 8, 256 threads, two CTAs per SM, table in shared memory
//           (n <= 16384), except R = 16, 512 threads where R = 8 would need
//           exactly 8 or 16 CTAs; R = 8, 512 threads (n <= 32768); R = 4, 512
//           threads, table read through L1 (n <= 65536); R = 16 on request.
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
  // measured on GB300: where 8-wide tiles need exactly 8 or 16 CTAs, 16-wide
  // tiles of 512 threads (the same blocks per CTA, half the tiles, so half the
  // exchanges per right-hand side) are 3-8% faster; elsewhere 2-5% slower
  if (t == 32 && fits(cand[0]) && (sh.C == 8 || sh.C == 16) && fits(kCand32[3])) return true;
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
  if (one) {
    L.one = *one;
    L.one.m = sh.m;
    L.one.g = sh.C;
  }
  L.nitems = nitems;
  L.single = items ? 0 : 1;
  L.m = sh.m;
  L.C = sh.C;
  L.err = err;
  tdm_status st = TDM_OK;
  if (!with_shape(sh, t, [&](auto tag) {
        using S = decltype(tag);
        const int maxc = shape_max_clusters<S, kLaunchSingle>(sh);
        if (items) st = launch_shape<S, kLaunchList>(sh, L, nitems < maxc ? nitems : maxc, s);
        else st = launch_shape<S, kLaunchSingle>(sh, L, nitems < maxc ? nitems : maxc, s);
      }))
    return TDM_ERR_NOT_IMPLEMENTED;
  return st;
}

tdm_status tdm_refined_launch_grouped(const RefShape& sh, int t, const RefItem* items, const int* units,
                                      const int* ustart, int nclusters, int* err, cudaStream_t s) {
  if (nclusters <= 0) return TDM_OK;
  RefLaunch L;
  memset(&L, 0, sizeof(L));
  L.items = items;
  L.units = units;
  L.ustart = ustart;
  L.single = 0;
  L.m = sh.m;
  L.C = sh.C;
  L.err = err;
  tdm_status st = TDM_OK;
  if (!with_shape(sh, t, [&](auto tag) { st = launch_shape<decltype(tag), kLaunchGrouped>(sh, L, nclusters, s); }))
    return TDM_ERR_NOT_IMPLEMENTED;
  return st;
}

int tdm_refined_coop_grid(const RefShape& sh, int t) {
  int grid = 0;
  with_shape(sh, t, [&](auto tag) {
    using S = decltype(tag);
    auto kern = refined_kernel<S, kLaunchCoop>();
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, sh.threads, sh.smem) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    grid = (nb * sms / sh.C) * sh.C;
  });
  return grid;
}

size_t tdm_refined_coop_scratch(const RefShape& sh, int grid) { return sizeof(float) * (size_t)grid * kScr(sh.R); }

int tdm_refined_coop_choice(const RefShape& sh, int t) {
  if (sh.C < 2) return 0;
  int slots = 0;
  if (!with_shape(sh, t, [&](auto tag) { slots = shape_max_clusters<decltype(tag), kLaunchSingle>(sh) * sh.C; }))
    return 0;
  const int grid = tdm_refined_coop_grid(sh, t);
  return (double)grid >= kCoopGain * (double)slots ? grid : 0;
}

tdm_status tdm_refined_launch_coop(const RefShape& sh, int t, const RefItem& one, int ntiles, int* err, float* scr,
                                   unsigned* ctr, int grid, cudaStream_t s) {
  if (ntiles <= 0) return TDM_OK;
  RefLaunch L;
  memset(&L, 0, sizeof(L));
  L.one = one;
  L.one.m = sh.m;
  L.one.g = sh.C;
  L.nitems = ntiles;
  L.single = 1;
  L.m = sh.m;
  L.C = sh.C;
  L.err = err;
  L.scr = scr;
  L.ctr = ctr;
  // no more groups than tiles
  const int groups = std::min(grid / sh.C, ntiles);
  TDM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned) * 32 * groups, s));
  tdm_status st = TDM_OK;
  if (!with_shape(sh, t, [&](auto tag) {
        using S = decltype(tag);
        auto kern = refined_kernel<S, kLaunchCoop>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess) {
          st = TDM_ERR_CUDA;
          return;
        }
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        lc.gridDim = dim3(groups * sh.C);
        lc.blockDim = dim3(sh.threads);
        lc.dynamicSmemBytes = sh.smem;
        lc.stream = s;
        lc.attrs = at;
        lc.numAttrs = 1;
        if (cudaLaunchKernelEx(&lc, kern, L) != cudaSuccess) st = TDM_ERR_CUDA;
      }))
    return TDM_ERR_NOT_IMPLEMENTED;
  return st;
}

int tdm_refined_coop_runs_grid(const RefShape& sh, int t) {
  int grid = 0;
  with_shape(sh, t, [&](auto tag) {
    using S = decltype(tag);
    auto kern = refined_kernel<S, kLaunchCoopRuns>();
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, sh.threads, sh.smem) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    grid = nb * sms;
  });
  return grid;
}

tdm_status tdm_refined_launch_coop_runs(const RefShape& sh, int t, const RefItem* items, const RefRun* runs,
                                        const int* rlist, const int* rstart, int nruns, int grid, float* scr,
                                        unsigned* ctr, int* err, cudaStream_t s) {
  if (nruns <= 0 || grid <= 0) return TDM_OK;
  RefLaunch L;
  memset(&L, 0, sizeof(L));
  L.items = items;
  L.units = rlist;
  L.ustart = rstart;
  L.runs = runs;
  L.single = 0;
  L.m = sh.m;
  L.C = 1;
  L.err = err;
  L.scr = scr;
  L.ctr = ctr;
  TDM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned) * 32 * (size_t)nruns, s));
  tdm_status st = TDM_OK;
  if (!with_shape(sh, t, [&](auto tag) {
        using S = decltype(tag);
        auto kern = refined_kernel<S, kLaunchCoopRuns>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess) {
          st = TDM_ERR_CUDA;
          return;
        }
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        lc.gridDim = dim3(grid);
        lc.blockDim = dim3(sh.threads);
        lc.dynamicSmemBytes = sh.smem;
        lc.stream = s;
        lc.attrs = at;
        lc.numAttrs = 1;
        if (cudaLaunchKernelEx(&lc, kern, L) != cudaSuccess) st = TDM_ERR_CUDA;
      }))
    return TDM_ERR_NOT_IMPLEMENTED;
  return st;
}

int tdm_refined_max_clusters(const RefShape& sh, int t) {
  int maxc = 0;
  if (!with_shape(sh, t, [&](auto tag) { maxc = shape_max_clusters<decltype(tag), kLaunchGrouped>(sh); })) return 0;
  return maxc;
}

RefItem tdm_refined_item(const tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                         int series, const RefShape& sh) {
  RefItem it;
  memset(&it, 0, sizeof(it));
  it.m = sh.m;
  it.g = sh.C;
  it.F = F; it.X = X; it.ldF = ldF; it.ldX = ldX;
  it.tab = p->rtab; it.rR = p->rR; it.rL = p->rL;
  it.n = (int)p->n; it.M = p->M; it.N = (int)N; it.tile = 0;
  it.series = series;
  it.steps = p->refine_steps;
  it.contraction = p->contraction;
  return it;
}

tdm_status tdm_launch_refined(tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                              cudaStream_t s, bool allow_coop) {
  if (ldF > kRefMaxLd || ldX > kRefMaxLd) return TDM_ERR_NOT_IMPLEMENTED;
  RefShape sh;
  if (!tdm_refined_shape(p->M, p->t, p->tile_rhs, sh)) return TDM_ERR_NOT_IMPLEMENTED;
  const RefItem one = tdm_refined_item(p, F, ldF, X, ldX, N, 0, sh);
  const int ntiles = (int)((N + sh.R - 1) / sh.R);
  if (allow_coop && p->coop_grid > 0)
    return tdm_refined_launch_coop(sh, p->t, one, ntiles, p->dev_err, p->coop_scr, p->coop_ctr, p->coop_grid, s);
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
