// tdm_prepare.cu -- the preliminary step of Algorithms 3 and 4 (Sections 3.3-3.4),
// executed once per matrix, in binary64, on the GPU.
//
// Rows are cut into blocks of t rows; block b covers [b*t, min(b*t+t, n)) and,
// for b >= 1, starts with the separator row p_b = b*t.  The step computes
//
//  * the pivots of the sweep of A from the top (dF) and from the bottom (dB):
//      dF_0 = b_0,      dF_i = b_i - a_{i-1}^2 / dF_{i-1},
//      dB_{n-1} = b_{n-1}, dB_i = b_i - a_i^2 / dB_{i+1};
//    their ratios -a_i/dF_i and -a_{i-1}/dB_i are the sweep coefficients of the
//    homogeneous problems B^L_k Z = e^L and B^R_k Z = e^R of eq. z_vector
//    (the alpha_i of the proof of Theorem 4);
//  * for every separator k the inverse row G_k = A^{-1} e_k (eq. green_v;
//    column = row by Lemma 2) on the two blocks next to it.  Its diagonal is
//    G_k(k) = 1 / (dF_k - a_k^2 / dB_{k+1}), and away from k it follows the
//    homogeneous solutions: G_k(i) = -a_i/dF_i * G_k(i+1) for i < k and
//    G_k(i) = -a_{i-1}/dB_i * G_k(i-1) for i > k;
//  * the ratios between neighbouring separators used by Theorem 2,
//      rR_q = Z^R_{p_q}(p_{q+1}) = prod_{i=p_q+1}^{p_{q+1}} (-a_{i-1}/dB_i),
//      rL_q = Z^L_{p_q}(p_{q-1}) = prod_{i=p_{q-1}}^{p_q - 1} (-a_i/dF_i);
//  * for every block interior the local sweep (Lemma 1: the interior with both
//    separator values known is an independent Dirichlet problem) and the
//    interior's responses phiL, phiR to unit separator values;
//  * checks: vanishing pivots (nondegeneracy, Section 2) and diagonal
//    dominance (Theorem 4), plus the largest |rR|, |rL| and the smallest pivot.
//
// The pivots, the inverse rows and the ratios are carried in double-double
// arithmetic and rounded to binary64 once.  In binary64 alone the pivot
// recurrence and the cancellation in 1/(dF_k - a_k^2/dB_{k+1}) leave the
// inverse rows of an ill-conditioned matrix (kappa ~ 1e6) only ~1e-12
// accurate, and the separator values of Theorem 2 inherit that error
// multiplied by sum |G_k(i) F_i| / |x_k|, which is large for oscillating F.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tdm_dd.cuh"
#include "tdm_internal.cuh"
#include "tdm_refine.cuh"

namespace {

__device__ __forceinline__ void atomic_max_pos(unsigned long long* slot, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_pos(unsigned long long* slot, double v) {
  atomicMin(slot, (unsigned long long)__double_as_longlong(v));
}

// stat[0]: flag bits; stat[1]: max |A| row sum; stat[2]: min |pivot|; stat[3]: max |z ratio|
__global__ void k_norm_and_dominance(const double* __restrict__ a, const double* __restrict__ b,
                                     int64_t n, unsigned long long* stat) {
  double rmax = 0.0;
  unsigned flags = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double al = (i > 0) ? fabs(a[i - 1]) : 0.0;
    const double ar = (i + 1 < n) ? fabs(a[i]) : 0.0;
    const double bi = fabs(b[i]);
    if (!isfinite(bi) || !isfinite(al) || !isfinite(ar)) flags |= kStatNonFinite;
    rmax = fmax(rmax, bi + al + ar);
    if (bi < al + ar) flags |= kStatNotDominant;
    if (bi > al + ar) flags |= kStatStrict;
  }
  if (flags) atomicOr(&stat[0], (unsigned long long)flags);
  atomic_max_pos(&stat[1], rmax);
}

// Pivots of the sweep of A from the top (block 0: dF_i = b_i - a_{i-1}^2 / dF_{i-1})
// and from the bottom (block 1: dB_i = b_i - a_i^2 / dB_{i+1}), in double-double.
// A step d -> b - a^2 / d is linear fractional: with d = p / q it is
// (p, q) -> (b p - a^2 q, p), a 2x2 matrix.  The rows are cut into one chunk per
// thread; each thread multiplies its chunk's matrices (no division; rescaled
// by powers of two, which leaves p / q unchanged), one thread carries the
// state through the chunk products to find every chunk's incoming pivot, and
// every thread then runs the recurrence itself over its chunk.
struct dd2x2 {
  dd m00, m01, m10, m11;
};
__device__ __forceinline__ void mob_step(dd2x2& C, double bi, dd a2) {   // C <- [[b, -a^2], [1, 0]] C
  const dd n00 = dd_sub(dd_mul_d(C.m00, bi), dd_mul(a2, C.m10));
  const dd n01 = dd_sub(dd_mul_d(C.m01, bi), dd_mul(a2, C.m11));
  C.m10 = C.m00;
  C.m11 = C.m01;
  C.m00 = n00;
  C.m01 = n01;
}
__device__ __forceinline__ dd dd_scale(dd x, double s) { return dd{x.hi * s, x.lo * s}; }   // s a power of two
__device__ __forceinline__ double pow2_near_inverse(double mx) {
  int e;
  frexp(mx, &e);
  return ldexp(1.0, -e);
}
__device__ __forceinline__ void mob_rescale(dd2x2& C) {
  const double mx = fmax(fmax(fabs(C.m00.hi), fabs(C.m01.hi)), fmax(fabs(C.m10.hi), fabs(C.m11.hi)));
  if (mx > 0x1p+256 || (mx > 0.0 && mx < 0x1p-256)) {
    const double s = pow2_near_inverse(mx);
    C.m00 = dd_scale(C.m00, s); C.m01 = dd_scale(C.m01, s);
    C.m10 = dd_scale(C.m10, s); C.m11 = dd_scale(C.m11, s);
  }
}

constexpr int kPivotThreads = 256;

__global__ void __launch_bounds__(kPivotThreads) k_pivots(const double* __restrict__ a, const double* __restrict__ b,
                                                          int64_t n, dd* __restrict__ dF, dd* __restrict__ dB,
                                                          unsigned long long* stat) {
  __shared__ dd2x2 chunk[kPivotThreads];
  __shared__ dd sp[kPivotThreads], sq[kPivotThreads];
  const bool fwd = blockIdx.x == 0;
  const int T = blockDim.x, t = threadIdx.x;
  const double normA = __longlong_as_double((long long)stat[1]);
  const double tiny = 64.0 * 1.1102230246251565e-16 * normA;
  // step k (0 .. n-2) produces the pivot of row fwd ? k + 1 : n - 2 - k with a = a[fwd ? k : n - 2 - k]
  const int64_t steps = n - 1;
  const int64_t Q = (steps + T - 1) / T;
  const int64_t k0 = (int64_t)t * Q < steps ? (int64_t)t * Q : steps;
  const int64_t k1 = k0 + Q < steps ? k0 + Q : steps;
  dd2x2 C{dd_make(1.0), dd_make(0.0), dd_make(0.0), dd_make(1.0)};
  for (int64_t k = k0; k < k1; k++) {
    const int64_t ia = fwd ? k : n - 2 - k;
    mob_step(C, b[fwd ? k + 1 : n - 2 - k], two_prod(a[ia], a[ia]));
    if ((k - k0) % 16 == 15) mob_rescale(C);
  }
  mob_rescale(C);
  chunk[t] = C;
  __syncthreads();
  if (t == 0) {   // the state entering every chunk
    dd p = dd_make(b[fwd ? 0 : n - 1]), q = dd_make(1.0);
    for (int u = 0; u < T; u++) {
      sp[u] = p;
      sq[u] = q;
      const dd2x2 M = chunk[u];
      const dd np = dd_add(dd_mul(M.m00, p), dd_mul(M.m01, q));
      const dd nq = dd_add(dd_mul(M.m10, p), dd_mul(M.m11, q));
      const double mx = fmax(fabs(np.hi), fabs(nq.hi));
      const double sc = (mx > 0x1p+256 || (mx > 0.0 && mx < 0x1p-256)) ? pow2_near_inverse(mx) : 1.0;
      p = dd_scale(np, sc);
      q = dd_scale(nq, sc);
    }
  }
  __syncthreads();
  double dmin = INFINITY;
  bool bad = false;
  dd* out = fwd ? dF : dB;
  if (t == 0) {
    const double d0 = b[fwd ? 0 : n - 1];
    out[fwd ? 0 : n - 1] = dd_make(d0);
    dmin = fabs(d0);
    bad = !isfinite(d0);
  }
  if (k0 < k1) {
    dd d = dd_div(sp[t], sq[t]);   // the pivot of the row before the chunk
    for (int64_t k = k0; k < k1; k++) {
      const int64_t ia = fwd ? k : n - 2 - k;
      const int64_t row = fwd ? k + 1 : n - 2 - k;
      d = dd_sub(dd_make(b[row]), dd_div(two_prod(a[ia], a[ia]), d));
      out[row] = d;
      if (!isfinite(d.hi)) bad = true;
      else dmin = fmin(dmin, fabs(d.hi));
    }
  }
  if (bad || !(dmin > tiny)) atomicOr(&stat[0], (unsigned long long)kStatSingular);
  if (dmin < INFINITY) atomic_min_pos(&stat[2], dmin);
}

template <typename T>
__device__ __forceinline__ void store_row(T* dst, const double* v) {
#pragma unroll
  for (int k = 0; k < kNCOEF; k++) dst[k] = (T)v[k];
}

// One thread per block b.
// Nonsymmetric A (Section 3.5): the similarity T = diag(t), t_{k+1} = t_k
// (sub_k / sup_k)^(1/2), makes T^-1 A T symmetric with off-diagonal
// sign(sup_k) (sub_k sup_k)^(1/2), provided every sub_k sup_k > 0.  Only the
// ratios t_{k+1} / t_k are kept: the coefficients need t over one block at a
// time, never its running product over the whole matrix.
__global__ void k_symmetrize(const double* __restrict__ sub, const double* __restrict__ sup, int64_t n,
                             double* __restrict__ ahat, double* __restrict__ tr, unsigned long long* stat) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n - 1;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double c = sub[k], a = sup[k], p = c * a;
    if (!(p > 0.0) || !isfinite(p)) {
      atomicOr(&stat[0], (unsigned long long)kStatNotSymmetrizable);
      ahat[k] = 0.0;
      tr[k] = 1.0;
      continue;
    }
    ahat[k] = copysign(sqrt(p), a);
    tr[k] = sqrt(c / a);
  }
}

__global__ void k_block_coefficients(const double* __restrict__ a, const double* __restrict__ b,
                                     int64_t n, int t, int M,
                                     const dd* __restrict__ dF, const dd* __restrict__ dB,
                                     double* __restrict__ coef64, float* __restrict__ coef32,
                                     double* __restrict__ rR, double* __restrict__ rL,
                                     const double* __restrict__ tr, unsigned long long* stat) {
  const int bidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (bidx >= M) return;
  const double normA = __longlong_as_double((long long)stat[1]);
  const double tiny = 64.0 * 1.1102230246251565e-16 * normA;
  const int64_t lo = (int64_t)bidx * t;
  const int64_t hi = (lo + t < n) ? lo + t : n;     // exclusive
  const bool has_left = bidx >= 1;                  // separator at row lo
  const bool has_right = hi < n;                    // separator at row hi
  bool bad = false;
  double zmax = 0.0;
  double dmin = INFINITY;

  // local arrays are small: t <= 64
  double gR[64], gL[64], lf[64], invd[64], cc[64], phL[64], phR[64];
  for (int i = 0; i < hi - lo; i++) {
    gR[i] = gL[i] = lf[i] = invd[i] = cc[i] = phL[i] = phR[i] = 0.0;
  }

  // inverse-row diagonal at separator k: 1 / (dF_k - a_k^2 / dB_{k+1})
  auto gdiag = [&](int64_t k) -> dd {
    dd den = dF[k];
    if (k + 1 < n) den = dd_sub(den, dd_div(two_prod(a[k], a[k]), dB[k + 1]));
    if (!(fabs(den.hi) > 0.0) || !isfinite(den.hi)) { bad = true; return dd_make(0.0); }
    return dd_div(dd_make(1.0), den);
  };
  auto ratio_up = [&](int64_t i) -> dd { return dd_div(dd_make(-a[i]), dF[i]); };        // G(i)/G(i+1), i < k
  auto ratio_dn = [&](int64_t i) -> dd { return dd_div(dd_make(-a[i - 1]), dB[i]); };    // G(i)/G(i-1), i > k

  if (has_right) {   // G_{hi}(i) for i = hi-1 .. lo
    dd g = gdiag(hi);
    for (int64_t i = hi - 1; i >= lo; i--) {
      g = dd_mul(g, ratio_up(i));
      gR[i - lo] = dd_to_d(g);
    }
  }
  if (has_left) {    // G_{lo}(i) for i = lo .. hi-1
    dd g = gdiag(lo);
    gL[0] = dd_to_d(g);
    for (int64_t i = lo + 1; i < hi; i++) {
      g = dd_mul(g, ratio_dn(i));
      gL[i - lo] = dd_to_d(g);
    }
  }
  if (has_left && has_right) {
    dd zr = dd_make(1.0), zl = dd_make(1.0);
    for (int64_t i = lo + 1; i <= hi; i++) zr = dd_mul(zr, ratio_dn(i));
    for (int64_t i = lo; i <= hi - 1; i++) zl = dd_mul(zl, ratio_up(i));
    rR[bidx] = dd_to_d(zr);        // separator q = bidx (row lo) -> q+1 (row hi)
    rL[bidx + 1] = dd_to_d(zl);    // separator q = bidx+1 (row hi) -> q-1 (row lo)
    zmax = fmax(fabs(rR[bidx]), fabs(rL[bidx + 1]));
  }

  // local sweep of the interior [f, hi-1]
  const int64_t f = has_left ? lo + 1 : lo;
  const int64_t last = hi - 1;
  if (f <= last) {
    double d = b[f];
    for (int64_t i = f; i <= last; i++) {
      if (i > f) {
        const double l = a[i - 1] / d;
        lf[i - lo] = l;
        d = b[i] - l * a[i - 1];
      }
      if (!(fabs(d) > tiny) || !isfinite(d)) bad = true;
      dmin = fmin(dmin, fabs(d));
      invd[i - lo] = 1.0 / d;
      cc[i - lo] = (i < last) ? a[i] : 0.0;
    }
    if (has_left) {  // A_I phiL = -a_lo e_first
      double g = -a[lo];
      phL[f - lo] = g;   // forward values stored temporarily
      for (int64_t i = f + 1; i <= last; i++) { g = -lf[i - lo] * g; phL[i - lo] = g; }
      double y = 0.0;
      for (int64_t i = last; i >= f; i--) { y = (phL[i - lo] - cc[i - lo] * y) * invd[i - lo]; phL[i - lo] = y; }
    }
    if (has_right) { // A_I phiR = -a_last e_last
      double y = -a[last] * invd[last - lo];
      phR[last - lo] = y;
      for (int64_t i = last - 1; i >= f; i--) { y = -cc[i - lo] * y * invd[i - lo]; phR[i - lo] = y; }
    }
  }
  if (has_left) {    // separator row: value comes from the separator recurrences
    lf[0] = 0.0; invd[0] = 0.0; cc[0] = 0.0; phL[0] = 1.0; phR[0] = 0.0;
  }

  // Nonsymmetric A = T S T^-1 with S the symmetric matrix above: x = A^-1 F =
  // T S^-1 (T^-1 F).  Every factor of T folds into the coefficients as a ratio
  // of t within this block (P[i] = t_i / t_lo, Q[i] = t_hi / t_i), so that the
  // kernels solve A directly:
  //   beta weights   gR *= t_hi / t_i,  gL *= t_lo / t_i
  //   local sweep    lf *= t_i / t_{i-1},  cc *= t_i / t_{i+1}   (invd unchanged)
  //   responses      phL *= t_i / t_lo,  phR *= t_i / t_hi
  //   ratios         rR[q] *= t_hi / t_lo,  rL[q+1] *= t_lo / t_hi
  // (the separator values are then those of x, not of T^-1 x).
  if (tr) {
    double P[65], Q[65];
    const int nb = (int)(hi - lo);            // rows of the block
    const int ext = has_right ? nb + 1 : nb;  // with the right separator row
    P[0] = 1.0;
    for (int k = 1; k < ext; k++) P[k] = P[k - 1] * tr[lo + k - 1];
    Q[ext - 1] = 1.0;
    for (int k = ext - 2; k >= 0; k--) Q[k] = Q[k + 1] * tr[lo + k];
    for (int k = 0; k < nb; k++) {
      const int64_t i = lo + k;
      if (has_right) { gR[k] *= Q[k]; phR[k] /= Q[k]; }
      if (has_left) { gL[k] /= P[k]; phL[k] *= P[k]; }
      if (k > 0) lf[k] *= tr[i - 1];
      if (i + 1 < n) cc[k] /= tr[i];
    }
    if (has_left && has_right) {
      rR[bidx] *= Q[0];
      rL[bidx + 1] /= Q[0];
      zmax = fmax(fabs(rR[bidx]), fabs(rL[bidx + 1]));
    }
  }

  for (int64_t i = lo; i < hi; i++) {
    const int k = (int)(i - lo);
    double row[kNCOEF];
    row[kGR] = gR[k]; row[kGL] = gL[k]; row[kLF] = lf[k]; row[3] = 0.0;
    row[kC] = cc[k]; row[kINVD] = invd[k]; row[kPHIL] = phL[k]; row[kPHIR] = phR[k];
    for (int c = 0; c < kNCOEF; c++)
      if (!isfinite(row[c])) bad = true;
    store_row(coef64 + i * kNCOEF, row);
    store_row(coef32 + i * kNCOEF, row);
  }
  if (bad) atomicOr(&stat[0], (unsigned long long)kStatSingular);
  if (isfinite(dmin)) atomic_min_pos(&stat[2], dmin);
  atomic_max_pos(&stat[3], zmax);
}

// Residual coefficients: sigma_i = b_i + a_{i-1} + a_i formed exactly as a
// double-double (two error-free sums), then sigma and a_i split into three
// binary32 parts each.
__device__ __forceinline__ void two_sum(double x, double y, double& s, double& e) {
  s = x + y;
  const double z = s - x;
  e = (x - (s - z)) + (y - z);
}
__device__ __forceinline__ void split3(double hi, double lo, float* out) {
  const float p0 = (float)hi;
  const double r = (hi - (double)p0) + lo;
  const float p1 = (float)r;
  const float p2 = (float)(r - (double)p1);
  out[0] = p0; out[1] = p1; out[2] = p2;
}
__global__ void k_residual_coefficients(const double* __restrict__ a, const double* __restrict__ b,
                                        int64_t n, float* __restrict__ res32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double al = (i > 0) ? a[i - 1] : 0.0;
    const double ar = (i + 1 < n) ? a[i] : 0.0;
    double s1, e1, s2, e2;
    two_sum(b[i], al, s1, e1);
    two_sum(s1, ar, s2, e2);
    double sh, sl;
    two_sum(s2, e1 + e2, sh, sl);
    float out[kNRES] = {0, 0, 0, 0, 0, 0, 0, 0};
    float sg[3], av[3];
    split3(sh, sl, sg);
    split3(ar, 0.0, av);
    out[kS0] = sg[0]; out[kS1] = sg[1]; out[kS2] = sg[2];
    out[kA0] = av[0]; out[kA1] = av[1]; out[kA2] = av[2];
    for (int k = 0; k < kNRES; k++) res32[i * kNRES + k] = out[k];
  }
}

// The refined kernel's coefficient table (tdm_refine.cuh): every coefficient
// of rows j and j + t/2 side by side, phi also as a binary32 pair (its second
// word is phi - (float)phi, exact to binary64 rounding).
__global__ void k_refined_table(const double* __restrict__ coef64, const float* __restrict__ res32, int64_t n,
                                int t, int M, float* __restrict__ tab) {
  const int H = t / 2;
  const int64_t total = (int64_t)(M + 1) * (H + 1);   // H row pairs and the rest of every block
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(k / (H + 1)), j = (int)(k % (H + 1));
    float* blk = tab + (size_t)b * kRefTabStride(t);
    const int64_t row0 = (int64_t)b * t;
    if (j == H) {   // the local sweep row by row, and a of the row before the block
      for (int i = 0; i < t; i++) {
        const int64_t row = row0 + i;
        const bool ok = b < M && row < n;
        blk[kRefLF(t) + i] = ok ? (float)coef64[row * kNCOEF + kLF] : 0.f;
        const int w = t - 1 - i;   // the substitution's step that visits row i
        blk[kRefCI(t) + 2 * w] = ok ? (float)coef64[row * kNCOEF + kC] : 0.f;
        blk[kRefCI(t) + 2 * w + 1] = ok ? (float)coef64[row * kNCOEF + kINVD] : 0.f;
      }
      const int64_t prev = row0 - 1;
      const bool ok = b < M && prev >= 0 && prev < n;
      blk[kRefTail(t) + 0] = ok ? res32[prev * kNRES + kA0] : 0.f;
      blk[kRefTail(t) + 1] = ok ? res32[prev * kNRES + kA1] : 0.f;
      blk[kRefTail(t) + 2] = 0.f;
      blk[kRefTail(t) + 3] = 0.f;
      continue;
    }
    float v[kRefTP];
    for (int q = 0; q < kRefTP; q++) v[q] = 0.f;
    for (int h = 0; h < 2; h++) {
      const int64_t i = row0 + j + h * H;
      if (b >= M || i >= n) continue;
      const double* cr = coef64 + i * kNCOEF;
      const float* rr = res32 + i * kNRES;
      v[kRT_GR + h] = (float)cr[kGR];
      v[kRT_GL + h] = (float)cr[kGL];
      const float plh = (float)cr[kPHIL], prh = (float)cr[kPHIR];
      v[kRT_PLH + h] = plh;
      v[kRT_PRH + h] = prh;
      v[kRT_PLL + h] = (float)(cr[kPHIL] - (double)plh);
      v[kRT_PRL + h] = (float)(cr[kPHIR] - (double)prh);
      v[kRT_S0 + h] = rr[kS0];
      v[kRT_S1 + h] = rr[kS1];
      v[kRT_A0 + h] = rr[kA0];
      v[kRT_A1 + h] = rr[kA1];
    }
    for (int q = 0; q < kRefTP; q++) blk[j * kRefTP + q] = v[q];
  }
}

}  // namespace

static void tdm_free_plan(tdm_plan_s* p) {
  if (!p) return;
  cudaFree(p->coef64); cudaFree(p->coef32); cudaFree(p->res32); cudaFree(p->rtab);
  cudaFree(p->rR); cudaFree(p->rL); cudaFree(p->a64); cudaFree(p->b64); cudaFree(p->tr);
  cudaFree(p->piv); cudaFree(p->stat); cudaFree(p->dev_err); cudaFree(p->coop_scr); cudaFree(p->coop_ctr);
  cudaFree(p->coop64_scr); cudaFree(p->coop64_ctr);
  if (p->last) cudaEventDestroy(p->last);
  tdm_host_stage_free(p->host_stage);
  if (p->nseg > 0) tdm_free_large(p);
  delete p;
}

extern "C" tdm_status tdm_destroy(tdm_handle h) {
  if (!h) return TDM_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  if (h->last) cudaEventSynchronize(h->last);
  tdm_batched_forget(h);
  tdm_free_plan(h);
  (void)cudaGetLastError();   // leave no error behind for the next call
  cudaSetDevice(cur);
  return TDM_OK;
}

// ---------------------------------------------------------------------------
// Automatic refinement (refine_steps = 0): one solve of seeded right-hand sides
// with kRefineCalibSteps corrections records the size of every correction,
// max over columns of max|d_k| / max|x|.  Convergence is fast (each correction
// shrinks the error by the binary32 solve's relative accuracy), so the size of
// correction 2 per unit of correction 1 is the contraction of one correction:
// a property of the matrix and of the binary32 solve more than of F.  The plan
// then tests every tile of right-hand sides after its first correction with
// that contraction (estimated error = size of the first correction x the
// contraction) and after later ones with the ratio test (tdm_refine.cu).  Right-hand sides like the calibration's stop
// after one correction; ones whose first solve is far less accurate relative
// to their solution (pure high modes of an ill-conditioned matrix) take more.
// Plans too large for a cheap calibration keep contraction 1: at least two
// corrections per tile.
// ---------------------------------------------------------------------------
namespace {

// uniform pseudo-random values in [-1, 1) from an integer hash of the index
__global__ void k_calib_rhs(float* F, int64_t count, uint32_t seed) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)k * 2654435761u ^ seed;
    h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
    F[k] = (float)(int32_t)h * 4.656612873077393e-10f;
  }
}

constexpr int kRefineAdaptive = -1;   // per-tile test
constexpr size_t kCalibBytes = 256u << 20;

tdm_status calibrate_refinement(tdm_plan_s* p, cudaStream_t s) {
  p->refine_steps = kRefineAdaptive;
  int N = 64;
  while (N > 8 && (size_t)p->n * N * 12 > kCalibBytes) N /= 2;
  if ((size_t)p->n * N * 12 > kCalibBytes) return TDM_OK;
  RefShape sh;
  if (!tdm_refined_shape(p->M, p->t, p->tile_rhs, sh)) return TDM_OK;
  float* F = nullptr;
  double* X = nullptr;
  tdm_status st = TDM_OK;
  int h_err = 0;
  float ratios[kRefineCalibSteps] = {0.f, 0.f, 0.f, 0.f};
  if (cudaMalloc(&F, sizeof(float) * p->n * N) != cudaSuccess || cudaMalloc(&X, sizeof(double) * p->n * N) != cudaSuccess) {
    st = TDM_ERR_NO_MEMORY;
  } else {
    st = tdm_calibration_record(true, nullptr, s);
    cudaError_t e = cudaSuccess;
    if (st == TDM_OK) {
      k_calib_rhs<<<128, 256, 0, s>>>(F, p->n * N, 0x9e3779b9u);
      RefItem one = tdm_refined_item(p, F, N, X, N, N, 0, sh);
      one.steps = kRefineCalib;
      st = tdm_refined_launch(sh, p->t, nullptr, &one, (N + sh.R - 1) / sh.R, p->dev_err, s);
    }
    if (st == TDM_OK) st = tdm_calibration_record(false, ratios, s);
    if (st == TDM_OK) e = cudaMemcpyAsync(&h_err, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (st == TDM_OK && e == cudaSuccess) e = cudaMemsetAsync(p->dev_err, 0, sizeof(int), s);
    if (st == TDM_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st == TDM_OK && e != cudaSuccess) st = TDM_ERR_CUDA;
  }
  if (F) cudaFree(F);
  if (X) cudaFree(X);
  (void)cudaGetLastError();
  // ratios[k]: the size of correction k + 1
  if (st == TDM_OK && h_err == 0 && ratios[0] > 0.f && ratios[1] < ratios[0])
    p->contraction = ratios[1] / ratios[0];
  else if (st == TDM_OK && h_err == 0 && ratios[0] == 0.f)
    p->contraction = 0.f;   // the first solve was exact on the calibration columns
  return st;
}

}  // namespace

// The preparation of a symmetric matrix (a, b), or, with sub and sup, of a
// nonsymmetric one: then a is unused and the symmetrized off-diagonal is
// formed on the device.
static tdm_status prepare_plan(const double* a, const double* b, const double* sub, const double* sup, int64_t n,
                               const tdm_options* opt, void* stream, tdm_handle* out) {
  if (!out) return TDM_ERR_INVALID_ARG;
  *out = nullptr;
  const bool general = sub != nullptr || sup != nullptr;
  if (n < 1 || n > (int64_t(1) << 26) || !b) return TDM_ERR_INVALID_ARG;
  if (general ? (n > 1 && (!sub || !sup)) : (n > 1 && !a)) return TDM_ERR_INVALID_ARG;
  if (!tdm_aligned(b, 8) || (a && !tdm_aligned(a, 8)) || (sub && !tdm_aligned(sub, 8)) ||
      (sup && !tdm_aligned(sup, 8)))
    return TDM_ERR_INVALID_ARG;
  int t = 32, steps = 0, tile = 0;
  if (opt) {
    if (opt->flags != 0) return TDM_ERR_INVALID_ARG;
    if (opt->block_rows != 0) t = opt->block_rows;
    tile = opt->tile_rhs;
    if (opt->refine_steps != 0) steps = opt->refine_steps;
  }
  if (t != 16 && t != 32) return TDM_ERR_INVALID_ARG;
  if (steps < -1 || steps > 4) return TDM_ERR_INVALID_ARG;
  if (tile != 0 && tile != 4 && tile != 8 && tile != 16) return TDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();   // report only errors of this call

  tdm_plan_s* p = new tdm_plan_s();
  p->n = n;
  p->t = t;
  p->M = (int)((n + t - 1) / t);
  p->refine_steps = steps;
  p->tile_rhs = tile;
  p->general = general ? 1 : 0;
  cudaGetDevice(&p->device);
  const int64_t na = n > 1 ? n - 1 : 1;
  bool ok = cudaMalloc(&p->coef64, sizeof(double) * n * kNCOEF) == cudaSuccess &&
            cudaMalloc(&p->coef32, sizeof(float) * n * kNCOEF) == cudaSuccess &&
            cudaMalloc(&p->res32, sizeof(float) * n * kNRES) == cudaSuccess &&
            cudaMalloc(&p->rtab, sizeof(float) * (size_t)(p->M + 1) * kRefTabStride(t)) == cudaSuccess &&
            cudaMalloc(&p->rR, sizeof(double) * (p->M + 2)) == cudaSuccess &&
            cudaMalloc(&p->rL, sizeof(double) * (p->M + 2)) == cudaSuccess &&
            cudaMalloc(&p->a64, sizeof(double) * na) == cudaSuccess &&
            cudaMalloc(&p->b64, sizeof(double) * n) == cudaSuccess &&
            (!general || cudaMalloc(&p->tr, sizeof(double) * na) == cudaSuccess) &&
            cudaMalloc(&p->piv, sizeof(dd) * 2 * n) == cudaSuccess &&
            cudaMalloc(&p->stat, sizeof(unsigned long long) * 8) == cudaSuccess &&
            cudaMalloc(&p->dev_err, sizeof(int)) == cudaSuccess &&
            cudaEventCreateWithFlags(&p->last, cudaEventDisableTiming) == cudaSuccess;
  if (ok && !general) {   // a cooperative launch's scratch, where the rule prefers it to clusters
    RefShape sh;
    if (tdm_refined_shape(p->M, t, tile, sh) && sh.C > 1) {
      const int grid = tdm_refined_coop_choice(sh, t);
      if (grid > 0) {
        ok = cudaMalloc(&p->coop_scr, tdm_refined_coop_scratch(sh, grid)) == cudaSuccess &&
             cudaMalloc(&p->coop_ctr, sizeof(unsigned) * 32 * (grid / sh.C)) == cudaSuccess;
        p->coop_grid = grid;
      }
    }
    size_t scr64 = 0;
    const int grid64 = ok ? tdm_plain_coop_choice(p->M, t, &scr64) : 0;
    if (grid64 > 0) {
      ok = cudaMalloc(&p->coop64_scr, scr64) == cudaSuccess &&
           cudaMalloc(&p->coop64_ctr, sizeof(unsigned) * 32 * (size_t)grid64) == cudaSuccess;
      p->coop64_grid = grid64;
    }
  }
  if (!ok) {
    (void)cudaGetLastError();
    tdm_free_plan(p);
    return TDM_ERR_NO_MEMORY;
  }
  const double inf = INFINITY;
  unsigned long long init[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  memcpy(&init[2], &inf, sizeof(double));
  cudaError_t e = cudaSuccess;
  if (n > 1 && !general) e = cudaMemcpyAsync(p->a64, a, sizeof(double) * (n - 1), cudaMemcpyDeviceToDevice, s);
  else e = cudaMemsetAsync(p->a64, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->b64, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->stat, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->rR, 0, sizeof(double) * (p->M + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->rL, 0, sizeof(double) * (p->M + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dev_err, 0, sizeof(int), s);
  if (e == cudaSuccess && general && n > 1)
    k_symmetrize<<<(int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(sub, sup, n, p->a64, p->tr,
                                                                                          p->stat);
  if (e == cudaSuccess) {
    k_norm_and_dominance<<<64, 256, 0, s>>>(p->a64, p->b64, n, p->stat);
    k_pivots<<<2, kPivotThreads, 0, s>>>(p->a64, p->b64, n, reinterpret_cast<dd*>(p->piv), reinterpret_cast<dd*>(p->piv) + n, p->stat);
    k_block_coefficients<<<(p->M + 127) / 128, 128, 0, s>>>(
        p->a64, p->b64, n, t, p->M, reinterpret_cast<dd*>(p->piv), reinterpret_cast<dd*>(p->piv) + n, p->coef64, p->coef32, p->rR, p->rL,
        general && n > 1 ? p->tr : nullptr, p->stat);
    k_residual_coefficients<<<(int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(
        p->a64, p->b64, n, p->res32);
    {
      const int64_t rows = (int64_t)(p->M + 1) * (t / 2 + 1);
      k_refined_table<<<(int)((rows + 255) / 256 < 1024 ? (rows + 255) / 256 : 1024), 256, 0, s>>>(
          p->coef64, p->res32, n, t, p->M, p->rtab);
    }
    e = cudaGetLastError();
  }
  unsigned long long host_stat[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_stat, p->stat, sizeof(host_stat), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    tdm_free_plan(p);
    return TDM_ERR_CUDA;
  }
  const unsigned flags = (unsigned)host_stat[0];
  if (flags & kStatNotSymmetrizable) {   // Section 3.5 needs sub_k sup_k > 0
    tdm_free_plan(p);
    return TDM_ERR_INVALID_ARG;
  }
  double normA, dmin, zmax;
  memcpy(&normA, &host_stat[1], sizeof(double));
  memcpy(&dmin, &host_stat[2], sizeof(double));
  memcpy(&zmax, &host_stat[3], sizeof(double));
  p->max_abs_z = zmax;
  p->min_abs_pivot = normA > 0 ? dmin / normA : 0.0;
  p->dominant = (!(flags & kStatNotDominant) && (flags & kStatStrict)) ? 1 : 0;
  if (flags & (kStatSingular | kStatNonFinite)) {
    tdm_free_plan(p);
    return TDM_ERR_SINGULAR;
  }
  if (steps == 0 && !general) {
    const tdm_status st = calibrate_refinement(p, s);
    if (st != TDM_OK) {
      tdm_free_plan(p);
      return st;
    }
  }
  if (!general && n > (int64_t)1024 * t) {   // beyond one cluster: the two-level structure
    const tdm_status st = tdm_prepare_large(p, a, b, opt, s);
    if (st != TDM_OK) {
      (void)cudaGetLastError();
      tdm_free_plan(p);
      return st;
    }
  }
  *out = p;
  return TDM_OK;
}

extern "C" tdm_status tdm_prepare(const double* a, const double* b, int64_t n,
                                  const tdm_options* opt, void* stream, tdm_handle* out) {
  return prepare_plan(a, b, nullptr, nullptr, n, opt, stream, out);
}

extern "C" tdm_status tdm_prepare_general(const double* sub, const double* diag, const double* sup, int64_t n,
                                          const tdm_options* opt, void* stream, tdm_handle* out) {
  if (n > 1 && (!sub || !sup)) return TDM_ERR_INVALID_ARG;
  // n == 1 has no off-diagonal: a 1 x 1 general plan (sub, sup unused)
  static const double kNone = 0.0;
  return prepare_plan(nullptr, diag, n > 1 ? sub : &kNone, n > 1 ? sup : &kNone, n, opt, stream, out);
}
