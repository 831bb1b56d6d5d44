// tdm_refine.cu -- binary32 dichotomy solves with iterative refinement: F in
// binary32, X in binary64, accuracy of a binary64 solve (or better); one
// persistent kernel that serves a single series (tdm_solve) and many series of
// different sizes (tdm_solve_batched).
//
// Work items.  An item is one tile of R right-hand sides of one series
// A X = F.  A thread-block cluster processes one item at a time with all n rows
// (CTA c owns m blocks of t rows, thread (block, rhs) owns one block for one
// right-hand side) and walks a list of items; consecutive items of a cluster
// normally belong to the same series.  Per item:
//
//   x  = solve32(F)                                   (steps A2-A5, binary32)
//   repeat (adaptive, at most 4 times, or a fixed count):
//     r_i = F_i - (A x)_i                             (error-free, see below)
//     x  += solve32(r)
//   X_i = xh_i + xl_i rounded once to binary64.
//
// x is held as x0 + delta: x0, the first solve's binary32 result, in
// registers; delta, the sum of the corrections, in shared memory, updated with
// an exact TwoSum whose rounding error is carried to the output.  F is read
// from global memory for the first solve and again (from L2) for each
// residual, so shared memory holds no copy of the tile.
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
#include <vector>

#include "tdm_df.cuh"
#include "tdm_iface_df.cuh"
#include "tdm_kernel_common.cuh"
#include "tdm_refine.cuh"
#include "tdm_tma.cuh"

// Most corrections any tile of a per-tile-tested launch has made on this
// device since the counter was last cleared (read by the prepare-time
// calibration; concurrent launches can only raise it).
__device__ int g_tdm_corrections_max;

namespace {
using namespace tdmk;

// Estimated relative error left after a correction d_k: ratio_k^2 / ratio_{k-1}
// (linear convergence), with ratio_k = max over columns of max|d_k| / max|x|;
// after the first correction, ratio_1 itself.
constexpr float kRefineTol = 1e-12f;

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

// per-CTA, per-column maxima of |d| and |x0| into slot [2][R]: shuffles over
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

// streaming loads/stores for the right-hand sides and the solution: they are
// touched once per tile and must not evict the coefficients from L1
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_stream(double* p, double v) {
  asm volatile("st.global.cs.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void ldg4(const float* p, float& x, float& y, float& z, float& w) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  x = v.x; y = v.y; z = v.z; w = v.w;
}

// 4 coefficients from shared memory (SM = true) or through the read-only cache
template <bool SM>
__device__ __forceinline__ void cld4(const float* p, float& x, float& y, float& z, float& w) {
  if constexpr (SM) ld4(p, x, y, z, w);
  else ldg4(p, x, y, z, w);
}

// forward pass (A2 + A3)
template <int TT, bool FULL, bool SM>
__device__ __forceinline__ void forward_pass_g(float (&v)[TT], const float* cf, int nrows, float& bR, float& bL) {
  float g = 0.f;
#pragma unroll
  for (int i = 0; i < TT; i++) {
    if (FULL || i < nrows) {
      float gr, gl, lf, unused;
      cld4<SM>(cf + i * kNCOEF, gr, gl, lf, unused);
      bR = fmaf(gr, v[i], bR);
      bL = fmaf(gl, v[i], bL);
      g = fmaf(-lf, g, v[i]);
      v[i] = g;
    }
  }
}

// F of one block for one right-hand side (zero outside the system)
template <int TT, bool FULL>
__device__ __forceinline__ void load_rhs(float (&g)[TT], const float* Fp, int64_t ldF, bool active, int nrows) {
  if (active) {
#pragma unroll
    for (int i = 0; i < TT; i++) {
      g[i] = (FULL || i < nrows) ? ld_stream(Fp) : 0.f;
      Fp += ldF;
    }
  } else {
#pragma unroll
    for (int i = 0; i < TT; i++) g[i] = 0.f;
  }
}

// Residual r = F - A x of the iterate x = x0 + delta over one block, in
// row-sum form: r_i = F_i - sigma_i x_i + E_{i-1} - E_i with the fluxes
// E_i = a_i (x_{i+1} - x_i).  g holds F on entry and r on exit.  FIRST: delta
// is still zero (first correction), so the differences of x are single
// TwoSums and sigma x a pair-by-float product.  Rows past n carry zero
// coefficients, F and x, so they add nothing.  The rows are done in two parts
// so that the interior (rows 1 .. TT-2, this block's iterate only) can run
// while the cluster barrier that publishes the neighbours' edge values
// completes; rows 0 and TT-1 follow.

// r_i from F_i, the fluxes on both sides of row i and sigma_i x_i (the large
// fluxes cancel exactly in the first TwoSum)
__device__ __forceinline__ float residual_row(float Fi, f2pair Ep, f2pair E, f2pair S) {
  const f2pair w = two_sum_f(Ep.h, -E.h);
  const f2pair u = two_sum_f(Fi, w.h);
  const f2pair v = two_sum_f(u.h, -S.h);
  const float small = ((Ep.l - E.l) - S.l) + (w.l + u.l + v.l);
  return v.h + small;
}
template <bool FIRST>
__device__ __forceinline__ f2pair x_diff(f2pair x1, f2pair x0) {
  if constexpr (FIRST) return two_sum_f(x1.h, -x0.h);
  else return df_diff(x1, x0);
}
template <bool FIRST>
__device__ __forceinline__ f2pair sigma_x(float sh, float sl, f2pair x) {
  if constexpr (FIRST) return df_mul_f(f2pair{sh, sl}, x.h);
  else return df_mul(f2pair{sh, sl}, x);
}
template <int R, bool FIRST>
__device__ __forceinline__ f2pair x_at(const float* x0, const float* delta, int i) {
  return f2pair{x0[i], FIRST ? 0.f : delta[i * R]};
}

// rows 1 .. TT-2; returns E_0 and E_{TT-2} for the edge rows
template <int R, int TT, bool FULL, bool FIRST, bool SM, int RS>
__device__ __forceinline__ void residual_interior(float (&g)[TT], const float (&x0)[TT], const float* delta,
                                                  const float* rsb, int nrows, f2pair& E0, f2pair& Elast) {
  float sh, sl, ah = 0.f, al = 0.f;
  if (FULL || 0 < nrows) cld4<SM>(rsb, sh, sl, ah, al);   // kS0, kS1, kA0, kA1 of row 0
  f2pair xi = f2pair{x0[1], FIRST ? 0.f : delta[R]};
  f2pair Ep = df_mul(f2pair{ah, al}, x_diff<FIRST>(xi, f2pair{x0[0], FIRST ? 0.f : delta[0]}));
  E0 = Ep;
#pragma unroll
  for (int i = 1; i < TT - 1; i++) {
    sh = sl = ah = al = 0.f;
    if (FULL || i < nrows) cld4<SM>(rsb + i * RS, sh, sl, ah, al);
    const f2pair xn = f2pair{x0[i + 1], FIRST ? 0.f : delta[(i + 1) * R]};
    const f2pair E = df_mul(f2pair{ah, al}, x_diff<FIRST>(xn, xi));
    g[i] = residual_row(g[i], Ep, E, sigma_x<FIRST>(sh, sl, xi));
    Ep = E;
    xi = xn;
  }
  Elast = Ep;
}

// rows 0 and TT-1, with x at the rows just outside the block (xm, xp) and
// a_{row0-1} (aprev)
template <int R, int TT, bool FULL, bool FIRST, bool SM, int RS>
__device__ __forceinline__ void residual_edges(float (&g)[TT], const float (&x0)[TT], const float* delta,
                                               const float* rsb, int nrows, f2pair aprev, f2pair xm, f2pair xp,
                                               f2pair E0, f2pair Elast) {
  float sh = 0.f, sl = 0.f, ah = 0.f, al = 0.f;
  const f2pair x_first = f2pair{x0[0], FIRST ? 0.f : delta[0]};
  if (FULL || 0 < nrows) cld4<SM>(rsb, sh, sl, ah, al);
  const f2pair Em1 = df_mul(aprev, x_diff<FIRST>(x_first, xm));
  g[0] = residual_row(g[0], Em1, E0, sigma_x<FIRST>(sh, sl, x_first));
  sh = sl = ah = al = 0.f;
  if (FULL || TT - 1 < nrows) cld4<SM>(rsb + (TT - 1) * RS, sh, sl, ah, al);
  const f2pair x_last = f2pair{x0[TT - 1], FIRST ? 0.f : delta[(TT - 1) * R]};
  const f2pair E = df_mul(f2pair{ah, al}, x_diff<FIRST>(xp, x_last));
  g[TT - 1] = residual_row(g[TT - 1], Elast, E, sigma_x<FIRST>(sh, sl, x_last));
}

// A5 of a solve, in two parts.  The back substitution of the block's local
// sweep does not depend on the separator values, so it runs while the cluster
// barrier of A4 completes; y replaces g.
template <bool SM>
__device__ __forceinline__ void cld2(const float* p, float& x, float& y) {
  float2 v;
  if constexpr (SM) v = *reinterpret_cast<const float2*>(p);
  else v = __ldg(reinterpret_cast<const float2*>(p));
  x = v.x;
  y = v.y;
}
template <int TT, bool FULL, bool SM>
__device__ __forceinline__ void backward_y(float (&g)[TT], const float* cf, int nrows) {
  float y = 0.f;
#pragma unroll
  for (int i = TT - 1; i >= 0; i--) {
    if (FULL || i < nrows) {
      float cc, invd;
      cld2<SM>(cf + i * kNCOEF + kC, cc, invd);
      y = fmaf(-cc, y, g[i]) * invd;
      g[i] = y;
    }
  }
}
// Then the correction with the separator values, d = y + phiL xL + phiR xR,
// and the update of the iterate x = x0 + delta: x0 (registers) is the first
// solve's result, delta (shared memory, stride R) accumulates the corrections.
//   FIRST (the first solve): x0 = d, g = 0.
//   otherwise: d is added to delta with Knuth's TwoSum; its exact rounding
//   error replaces g[i], so that the output can include the last one.
// TRACK: maxd = max |d| over the block (for the convergence test).
template <int R, int TT, bool FULL, bool SM, bool FIRST, bool TRACK>
__device__ __forceinline__ void backward_d(float (&g)[TT], const float* cf, int nrows, float xL, float xR,
                                           float (&x0)[TT], float* delta, float& maxd) {
#pragma unroll
  for (int i = 0; i < TT; i++) {
    if (FULL || i < nrows) {
      float phl, phr;
      cld2<SM>(cf + i * kNCOEF + kPHIL, phl, phr);
      const float d = fmaf(phr, xR, fmaf(phl, xL, g[i]));
      if (FIRST) {
        x0[i] = d;
        g[i] = 0.f;
      } else {
        const f2pair sd = two_sum_f(delta[i * R], d);
        delta[i * R] = sd.h;
        g[i] = sd.l;
      }
      if (TRACK) maxd = fmaxf(maxd, fabsf(d));
    }
  }
}

template <int R, int TT, bool FULL, bool SM>
__device__ __forceinline__ void backward_d_any(bool first, bool track, float (&g)[TT], const float* cf, int nrows,
                                               float xL, float xR, float (&x0)[TT], float* delta, float& maxd) {
  if (first) backward_d<R, TT, FULL, SM, true, true>(g, cf, nrows, xL, xR, x0, delta, maxd);
  else if (track) backward_d<R, TT, FULL, SM, false, true>(g, cf, nrows, xL, xR, x0, delta, maxd);
  else backward_d<R, TT, FULL, SM, false, false>(g, cf, nrows, xL, xR, x0, delta, maxd);
}

// floats per block of the staged solve coefficients (16 bytes of padding)
template <int TT>
constexpr int kCfStride = TT * kNCOEF + 4;

// Shared-memory layout of the refined kernel (byte offsets; the same function
// sizes the launch on the host).
struct RefOffsets {
  size_t delta, edge, red, cvg, coef, res, pad, iface, bytes;
};
__host__ __device__ constexpr RefOffsets refine_offsets(int R, int TT, int NT, bool sm_coef) {
  const size_t MM = (size_t)(NT / R);
  RefOffsets o{};
  size_t p = 0;
  o.delta = p; p += round16(4 * MM * (TT + 1) * R);
  o.edge = p; p += round16(4 * 4 * MM * R);
  o.red = p; p += round16(4 * 2 * MM * R);
  o.cvg = p; p += round16(4 * 5 * (size_t)R);
  o.coef = p; if (sm_coef) p += round16(4 * MM * (TT * kNCOEF + 4));
  o.res = p; if (sm_coef) p += round16(16 * MM * (TT + 1));
  o.pad = p; if (sm_coef) p += round16(4 * (size_t)(TT + 1) * R);   // delta words of threads past the blocks
  o.iface = p; p += iface_offsets(R, (int)MM, true).bytes;
  o.bytes = p;
  return o;
}

template <int R, int TT, int NT, int MINB, bool SM>
__global__ void __launch_bounds__(NT, MINB) k_refined(const RefLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float ratio_s;
  constexpr int MM = NT / R;                               // most blocks a CTA can own
  constexpr RefOffsets O = refine_offsets(R, TT, NT, SM);
  const int m = L.m;
  const int rows_cta = m * TT;
  // Every array at a compile-time offset of the shared window.  Per-block
  // arrays carry one padding row (sxl, sres) or 16 bytes (scf) per block: the
  // 32 / R blocks a warp covers then fall in different banks.
  float* const sxl = reinterpret_cast<float*>(smem_raw + O.delta);   // [MM][TT+1][R] corrections delta
  float* const eFh = reinterpret_cast<float*>(smem_raw + O.edge);    // [4][MM][R] block edge values of x
  float* const eFl = eFh + MM * R;
  float* const eLh = eFl + MM * R;
  float* const eLl = eLh + MM * R;
  float* const redD = reinterpret_cast<float*>(smem_raw + O.red);    // [2][warps][R] per-warp maxima
  float* const cvg = reinterpret_cast<float*>(smem_raw + O.cvg);     // [2][2][R] per-CTA maxima, read remotely
  float* const cvg_scratch = cvg + 4 * R;                            // [R]
  // SM: the CTA's coefficient rows, reloaded when the series changes
  float* const scf = reinterpret_cast<float*>(smem_raw + O.coef);    // [MM][TT*8+4]
  float* const sres = reinterpret_cast<float*>(smem_raw + O.res);    // [MM][TT+1][4]
  const IfaceDF<R, MM> f{smem_raw + O.iface};
  const unsigned c = cluster_rank();
  const int tid = threadIdx.x;
  const int r = tid % R;
  const int bl = tid / R;
  const int cluster_id = blockIdx.x / L.C;
  const int nclusters = gridDim.x / L.C;
  // Threads past the CTA's blocks (bl >= m) only round the CTA up to whole
  // warps.  With staged coefficients they run the same full-block code on block
  // 0's coefficients and a scratch delta block, so that no per-row guard is
  // compiled in; every result they produce is discarded.
  const bool pad_thread = bl >= m;
  float* xlt = (SM && pad_thread) ? reinterpret_cast<float*>(smem_raw + O.pad) + r
                                  : sxl + (size_t)bl * (TT + 1) * R + r;   // this thread's delta words

  int cur_series = -1;
  int parity = 0;

  bool preloaded = false;   // g already holds this item's F (loaded during the previous output)
  for (int it = cluster_id; it < L.nitems; it += nclusters) {
    // fields of the current item, read where they are used (kernel parameter
    // or work list; no address of the parameter is taken)
#define ITEM(f) (L.single ? L.one.f : L.items[it].f)
    const int tile = L.single ? it : L.items[it].tile;
    if (ITEM(series) != cur_series) {   // new series: ratios and prefix products
      __syncthreads();
      iface_df_setup(f, ITEM(rR), ITEM(rL), ITEM(M), m, L.C, c);
      if constexpr (SM) {   // rows past n are staged as zeros
        const int64_t cta_row0 = (int64_t)c * rows_cta;
        for (int k = tid; k < rows_cta * kNCOEF / 4; k += blockDim.x) {
          const int rr = (k * 4) / kNCOEF;   // row within the CTA
          const int64_t row = cta_row0 + rr;
          float x = 0.f, y = 0.f, z = 0.f, w = 0.f;
          if (row < ITEM(n)) ldg4(ITEM(coef) + cta_row0 * kNCOEF + (int64_t)k * 4, x, y, z, w);
          float* d = scf + (size_t)(rr / TT) * kCfStride<TT> + (size_t)(rr % TT) * kNCOEF + (k * 4) % kNCOEF;
          d[0] = x; d[1] = y; d[2] = z; d[3] = w;
        }
        for (int k = tid; k < m * (TT + 1); k += blockDim.x) {   // block j: rows j*TT-1 .. j*TT+TT-1
          const int64_t row = cta_row0 + (int64_t)(k / (TT + 1)) * TT + (k % (TT + 1)) - 1;
          float x = 0.f, y = 0.f, z = 0.f, w = 0.f;
          if (row >= 0 && row < ITEM(n)) ldg4(ITEM(res) + row * kNRES, x, y, z, w);   // kS0, kS1, kA0, kA1
          float* d = sres + (size_t)k * 4;
          d[0] = x; d[1] = y; d[2] = z; d[3] = w;
        }
      }
      __syncthreads();
      cur_series = ITEM(series);
    }
    const int n = ITEM(n);
    const int b = (int)c * m + bl;
    const bool blk_ok = (bl < m) && (b < ITEM(M));
    const int64_t row0 = (int64_t)b * TT;
    const int nrows = blk_ok ? (int)((n - row0) < TT ? (n - row0) : TT) : 0;
    const int64_t col = (int64_t)tile * R + r;
    const bool col_ok = col < ITEM(N);
    const bool active = nrows > 0 && col_ok;   // this thread's rows and column exist
    const bool full_rows = nrows == TT;
    // Arithmetic over all TT rows: with staged coefficients the rows past n
    // are zeros (F, x and every coefficient), so only F and X need guards.
    const bool full = full_rows;   // (staged coefficients: the full-block code runs always)
    const int blc = (SM && pad_thread) ? 0 : bl;
    const float* Fp = ITEM(F) + row0 * ITEM(ldF) + col;
    // this block's coefficient rows (rsb[-RS] is the row before the block)
    const float* cfb = SM ? scf + (size_t)blc * kCfStride<TT> : ITEM(coef) + row0 * kNCOEF;
    const float* rsb = SM ? sres + (size_t)(blc * (TT + 1) + 1) * 4 : ITEM(res) + row0 * kNRES;
    constexpr int RS = SM ? 4 : kNRES;   // stride of the residual coefficient rows
    const bool adaptive = ITEM(steps) <= 0;
    const int cap = adaptive ? 4 : ITEM(steps);

    float xh[TT], g[TT];
#pragma unroll
    for (int i = 0; i < TT; i++) {
      xh[i] = 0.f;
      if (SM || bl < m) xlt[i * R] = 0.f;
    }
    if (!preloaded) {
      if (full_rows) load_rhs<TT, true>(g, Fp, ITEM(ldF), active, nrows);
      else load_rhs<TT, false>(g, Fp, ITEM(ldF), active, nrows);
    }
    bool have_f = false;   // g holds F for the next residual (loaded right after the last solve)

    float ratio_prev = 1.f;
    float maxx = 0.f;   // max |x0| of this thread's rows (the first solve)
    int cpar = 0;
    for (int step = 0;; step++) {
      if (step > 0) {
        // ---- residual r = F - A x of the current iterate ------------------------
        if (bl < m) {
          eFh[bl * R + r] = xh[0]; eFl[bl * R + r] = xlt[0];
          eLh[bl * R + r] = xh[TT - 1]; eLl[bl * R + r] = xlt[(TT - 1) * R];
        }
        // Adaptive refinement makes at least two corrections; from the third
        // step on it first tests the last one (estimated error
        // ratio_k^2 / ratio_{k-1}), which needs every CTA's maxima.  Otherwise
        // the interior of the residual overlaps the edge-value barrier.
        const bool test = adaptive && step >= 3;
        if (test) {
          cluster_barrier();
          if (step == 3) ratio_prev = cluster_ratio<R>(cvg + cpar * 2 * R, L.C, tid, cvg_scratch, &ratio_s);
          const float ratio = cluster_ratio<R>(cvg + (cpar ^ 1) * 2 * R, L.C, tid, cvg_scratch, &ratio_s);
          const bool stop = ratio * ratio <= kRefineTol * ratio_prev;
          ratio_prev = ratio;
          if (stop) {
            if (tid == 0 && c == 0) atomicMax(&g_tdm_corrections_max, step - 1);
            break;
          }
        } else {
          cluster_arrive();
        }
        f2pair E0{0.f, 0.f}, Elast{0.f, 0.f};
        if (bl < m) {
          if (!have_f) {
            if (full_rows) load_rhs<TT, true>(g, Fp, ITEM(ldF), active, nrows);
            else load_rhs<TT, false>(g, Fp, ITEM(ldF), active, nrows);
          }
          have_f = false;
          if (nrows > 0) {
            if (step == 1) {   // delta is still zero
              if (SM || full) residual_interior<R, TT, true, true, SM, RS>(g, xh, xlt, rsb, nrows, E0, Elast);
              else residual_interior<R, TT, SM, true, SM, RS>(g, xh, xlt, rsb, nrows, E0, Elast);
            } else {
              if (SM || full) residual_interior<R, TT, true, false, SM, RS>(g, xh, xlt, rsb, nrows, E0, Elast);
              else residual_interior<R, TT, SM, false, SM, RS>(g, xh, xlt, rsb, nrows, E0, Elast);
            }
          }
        }
        if (!test) cluster_wait();
        if (bl < m) {
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
          if (nrows > 0) {
            // a_{row0-1}, for the flux into the first row
            f2pair aprev{0.f, 0.f};
            if (row0 > 0) aprev = f2pair{rsb[-RS + kA0], rsb[-RS + kA1]};
            if (step == 1) {
              if (SM || full) residual_edges<R, TT, true, true, SM, RS>(g, xh, xlt, rsb, nrows, aprev, xm, xp, E0, Elast);
              else residual_edges<R, TT, SM, true, SM, RS>(g, xh, xlt, rsb, nrows, aprev, xm, xp, E0, Elast);
            } else {
              if (SM || full) residual_edges<R, TT, true, false, SM, RS>(g, xh, xlt, rsb, nrows, aprev, xm, xp, E0, Elast);
              else residual_edges<R, TT, SM, false, SM, RS>(g, xh, xlt, rsb, nrows, aprev, xm, xp, E0, Elast);
            }
          }
        }
      }
      // ---- binary32 dichotomy solve of g (A2-A5) ---------------------------------
      float bR = 0.f, bL = 0.f;
      if (SM || full) forward_pass_g<TT, true, SM>(g, cfb, nrows, bR, bL);
      else forward_pass_g<TT, SM, SM>(g, cfb, nrows, bR, bL);
      if (bl < m) {
        f.beR()[bl * f.kRP + r] = bR;
        f.beL()[bl * f.kRP + r] = bL;
      }
      __syncthreads();
      iface_df_scan<R>(f, m, parity);
      cluster_arrive();   // the back substitution overlaps the exchange of the CTA totals
      if (SM || full) backward_y<TT, true, SM>(g, cfb, nrows);
      else backward_y<TT, SM, SM>(g, cfb, nrows);
      cluster_wait();
      iface_df_fold<R>(f, L.C, c, parity);
      __syncthreads();
      parity ^= 1;
      float xL = 0.f, xR = 0.f;
      if (blk_ok) {
        if (b >= 1) xL = iface_df_sep<R>(f, bl, r);
        if (b + 1 <= ITEM(M) - 1) xR = iface_df_sep<R>(f, bl + 1, r);
      }
      float maxd = 0.f;
      const bool first = step == 0;
      if (SM || full) backward_d_any<R, TT, true, SM>(first, adaptive, g, cfb, nrows, xL, xR, xh, xlt, maxd);
      else backward_d_any<R, TT, SM, SM>(first, adaptive, g, cfb, nrows, xL, xR, xh, xlt, maxd);
      if (!col_ok) maxd = 0.f;   // padding columns of a ragged tile do not vote
      if (first) {
        maxx = maxd;
      } else if (adaptive) {   // per-CTA, per-column maxima of |d| and |x0| for the test
        cta_maxima<R>(maxd, maxx, redD, cvg + cpar * 2 * R, tid);
        cpar ^= 1;
      }
      // when another correction is certain, the last rounding errors in g are
      // not needed: reload F now, so that the loads overlap the bookkeeping
      // and the edge-value exchange
      if (step < cap && (!adaptive || step < 2) && bl < m) {
        if (full_rows) load_rhs<TT, true>(g, Fp, ITEM(ldF), active, nrows);
        else load_rhs<TT, false>(g, Fp, ITEM(ldF), active, nrows);
        have_f = true;
      }
      if (step == cap) {
        if (adaptive) {   // cap reached: record whether the last correction met the test
          cluster_barrier();
          if (step < 3) ratio_prev = step == 2 ? cluster_ratio<R>(cvg + cpar * 2 * R, L.C, tid, cvg_scratch, &ratio_s)
                                               : 1.f;
          const float ratio = cluster_ratio<R>(cvg + (cpar ^ 1) * 2 * R, L.C, tid, cvg_scratch, &ratio_s);
          if (tid == 0 && !(ratio * ratio <= kRefineTol * ratio_prev)) atomicExch(L.err, kDevErrNotConverged);
          if (tid == 0 && c == 0) atomicMax(&g_tdm_corrections_max, cap);
        }
        break;
      }
    }
    // ---- X = x0 + delta + (last rounding error, in g), rounded once to binary64 ----
    // Each row's g is free once the row is stored: the next item's F row is
    // loaded into it there, so that its latency overlaps the rest of the output.
    {
      const int it2 = it + nclusters;
      preloaded = it2 < L.nitems;
      const float* Fn = nullptr;
      int64_t ldn = 0;
      int nrows_n = 0;
      if (preloaded) {
#define ITEM2(f) (L.single ? L.one.f : L.items[it2].f)
        const int tile_n = L.single ? it2 : L.items[it2].tile;
        const int64_t col_n = (int64_t)tile_n * R + r;
        const int n_n = ITEM2(n);
        if ((bl < m) && (b < ITEM2(M)) && col_n < ITEM2(N)) {
          nrows_n = (int)((n_n - row0) < TT ? (n_n - row0) : TT);
          ldn = ITEM2(ldF);
          Fn = ITEM2(F) + row0 * ldn + col_n;
        }
#undef ITEM2
      }
      const int64_t ldX = ITEM(ldX);
      double* Xp = ITEM(X) + row0 * ldX + col;
#pragma unroll
      for (int i = 0; i < TT; i++) {
        if (active && (full_rows || i < nrows)) {
          const f2pair sx = two_sum_f(xh[i], xlt[i * R]);
          st_stream(Xp, tdm_f2d(sx.h) + tdm_f2d(sx.l + g[i]));
        }
        Xp += ldX;
        g[i] = i < nrows_n ? ld_stream(Fn + (int64_t)i * ldn) : 0.f;
      }
    }
  }
#undef ITEM
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

}  // namespace

// Tile shapes: R right-hand sides per tile, NT threads per CTA, m = NT / R
// blocks of t rows per CTA, up to 16 CTAs per cluster.
//   t = 16: R = 8, 512 threads, two CTAs per SM (64 registers), 1024 rows per
//           CTA (n <= 16384); R = 4 with 512 threads (2048 rows) or 1024
//           threads (4096 rows, n <= 65536), coefficients read through L1.
//   t = 32: R = 8, 256 threads, two CTAs per SM (128 registers, n <= 16384);
//           R = 8, 512 threads, one CTA per SM (n <= 32768); R = 4, 512
//           threads, coefficients read through L1 (n <= 65536); R = 16,
//           512 threads on request.
// A requested width (pref) is tried first; the rule's shapes follow.
bool tdm_refined_shape(int M, int t, int pref, RefShape& sh) {
  struct Cand { int R, NT; bool sm; };
  // the requested width first (16 exists for 32-row blocks only)
  const Cand want = {pref == 16 && t == 16 ? 0 : pref, pref == 8 && t == 32 ? 256 : 512, pref != 4};
  const Cand c16[4] = {{8, 512, true}, {4, 512, false}, {4, 1024, false}, {4, 1024, false}};
  const Cand c32[4] = {{8, 256, true}, {8, 512, true}, {4, 512, false}, {4, 512, false}};
  const Cand* rule = t == 16 ? c16 : c32;
  for (int k = pref ? -1 : 0; k < 4; k++) {
    const Cand* cand = k < 0 ? &want : rule;
    const int idx = k < 0 ? 0 : k;
    const int R = cand[idx].R, NT = cand[idx].NT;
    if (R != 4 && R != 8 && R != 16) continue;
    const int m_max = NT / R;
    const int C = (M + m_max - 1) / m_max;
    if (C > 16) continue;
    const int m = (M + C - 1) / C;
    sh.R = R; sh.NT = NT; sh.m = m; sh.C = C;
    sh.threads = ((m * R + 31) / 32) * 32;
    if (sh.threads < 96) sh.threads = 96;
    sh.sm_coef = cand[idx].sm;
    sh.smem = refine_offsets(R, t, NT, sh.sm_coef).bytes;
    if (sh.smem > 227 * 1024) continue;
    return true;
  }
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
    case 8 * 100000 + 512 * 10 + 1: return launch_shape<8, 16, 512, 2, true>(sh, L, nitems, s);
    case 4 * 100000 + 512 * 10 + 1: return launch_shape<4, 16, 512, 2, false>(sh, L, nitems, s);
    case 4 * 100000 + 1024 * 10 + 1: return launch_shape<4, 16, 1024, 1, false>(sh, L, nitems, s);
  }
  return TDM_ERR_NOT_IMPLEMENTED;
}

RefItem tdm_refined_item(const tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                         int series) {
  RefItem it;
  memset(&it, 0, sizeof(it));
  it.F = F; it.X = X; it.ldF = ldF; it.ldX = ldX;
  it.coef = p->coef32; it.res = p->res32; it.rR = p->rR; it.rL = p->rL;
  it.n = (int)p->n; it.M = p->M; it.N = (int)N; it.tile = 0;
  it.series = series;
  it.steps = p->refine_steps;
  return it;
}

tdm_status tdm_launch_refined(tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                              cudaStream_t s) {
  RefShape sh;
  if (!tdm_refined_shape(p->M, p->t, p->tile_rhs, sh)) return TDM_ERR_NOT_IMPLEMENTED;
  const RefItem one = tdm_refined_item(p, F, ldF, X, ldX, N, 0);
  const int ntiles = (int)((N + sh.R - 1) / sh.R);
  return tdm_refined_launch(sh, p->t, nullptr, &one, ntiles, p->dev_err, s);
}

// Clears / reads the corrections counter of the current device (calibration).
tdm_status tdm_corrections_counter(bool clear, int* value, cudaStream_t s) {
  if (clear) {
    const int zero = 0;
    TDM_CUDA_TRY(cudaMemcpyToSymbolAsync(g_tdm_corrections_max, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    TDM_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    TDM_CUDA_TRY(cudaMemcpyFromSymbolAsync(value, g_tdm_corrections_max, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    TDM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return TDM_OK;
}
