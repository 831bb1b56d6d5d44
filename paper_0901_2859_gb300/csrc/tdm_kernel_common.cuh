// tdm_kernel_common.cuh -- device pieces shared by the plain and the refined
// solve kernels: cluster primitives, the shared-memory layout, and step A4
// (separator values by Theorem 2, eq. theor_2) for one tile.
#pragma once

#include <stdint.h>

#include "tdm_internal.cuh"

namespace tdmk {

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Cluster-wide barrier.  Every thread arrives (release); warp 0 alone waits
// for the other CTAs while the remaining warps sleep in the CTA barrier, then
// they complete their own wait (acquire) on the already finished phase.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  if (threadIdx.x < 32) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  __syncthreads();
  if (threadIdx.x >= 32) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The two halves of a cluster barrier, for work that overlaps its completion:
// arrive after the writes the other CTAs will read (release), wait before
// reading theirs (acquire).  Every thread of every CTA executes both.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// load a double from the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ double ld_cluster_f64(const double* local, unsigned rank) {
  const unsigned laddr = (unsigned)__cvta_generic_to_shared(local);
  unsigned raddr;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(raddr) : "memory");
  return v;
}

__device__ __forceinline__ float ld_cluster_f32(const float* local, unsigned rank) {
  const unsigned laddr = (unsigned)__cvta_generic_to_shared(local);
  unsigned raddr;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(raddr) : "memory");
  return v;
}

struct SolveArgs {
  const void* F;
  void* X;
  int64_t ldF, ldX, N;
  const void* coef;
  const double* rR;
  const double* rL;
  int* err;
  int n, M, m, C, ntiles;
  int box_rows;   // TMA box height (divides m * t)
  double* scr;    // cooperative binary64 solve: every CTA's partials [2 parity][2 dir][R]
  unsigned* ctr;  // cooperative binary64 solve: the groups' barrier counters (zero at launch)
};

struct Smem {
  double* lr;      // [(m+1) R]  local SR partials LR
  double* ll;      // [(m+1) R]  local SL partials LL
  double* piR;     // [m+1]
  double* piL;     // [m+1]
  double* rRloc;   // [m+1]
  double* rLloc;   // [m+1]
  double* piRtot;  // [16]
  double* piLtot;  // [16]
  double* xch;     // [2 parity][2 dir][R]  read by the other CTAs
  double* in;      // [2][R]  incoming partials (binary64)
  float* piR32;    // [m+1]
  float* piL32;    // [m+1]
  float* in32;     // [2][R]
  double* betaR;   // [m R] beta^R of every block, converted to binary64 by its thread
  double* betaL;   // [m R]
};

__host__ __device__ inline size_t fbuf_bytes(int m, int t, int R, int tsize, bool tma) {
  return tma ? (size_t)m * t * R * tsize : 0;
}
constexpr int kCPAD = 4;   // elements after each block's coefficient rows (bank offset between blocks)
__host__ __device__ inline size_t coef_bytes(int m, int t, int tsize) {
  return (size_t)m * (t * kNCOEF + kCPAD) * tsize;
}
__host__ __device__ inline size_t smem_bytes(int m, int t, int R, int tsize, bool tma) {
  // interface arrays as laid out by carve(), each rounded up to 16 bytes
  const size_t d = 2 * (sizeof(double) * (m + 1) * R + 16) + 4 * (sizeof(double) * (m + 1) + 16) + 256 +
                   (sizeof(double) * 6 * R + 32);
  const size_t f = 2 * (sizeof(float) * (m + 1) + 16) + sizeof(float) * 2 * R + 16;
  const size_t tb = 2 * (sizeof(double) * m * R + 16);
  return 128 + fbuf_bytes(m, t, R, tsize, tma) + coef_bytes(m, t, tsize) + d + f + tb;
}

// 2 coefficients starting at p (8-byte aligned for binary32) in one vector load
__device__ __forceinline__ void ld2(const float* p, float& x, float& y) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  x = v.x; y = v.y;
}
__device__ __forceinline__ void ld2(const double* p, double& x, double& y) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  x = v.x; y = v.y;
}
// the 4 coefficients starting at p (16-byte aligned) in one or two vector loads
__device__ __forceinline__ void ld4(const float* p, float& x, float& y, float& z, float& w) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x = v.x; y = v.y; z = v.z; w = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& x, double& y, double& z, double& w) {
  const double2 v0 = *reinterpret_cast<const double2*>(p);
  const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
  x = v0.x; y = v0.y; z = v1.x; w = v1.y;
}

__host__ __device__ constexpr size_t round16(size_t x) { return (x + 15) & ~size_t(15); }

// Carves the interface arrays out of shared memory starting at p (16-byte
// aligned).  Pointers are derived from the __shared__ array by pointer
// arithmetic only, so the compiler keeps them in the shared address space.
__device__ inline Smem carve(unsigned char* p, int m, int R, int tsize) {
  Smem s;
  s.lr = reinterpret_cast<double*>(p); p += round16(sizeof(double) * (m + 1) * R);
  s.ll = reinterpret_cast<double*>(p); p += round16(sizeof(double) * (m + 1) * R);
  s.piR = reinterpret_cast<double*>(p); p += round16(sizeof(double) * (m + 1));
  s.piL = reinterpret_cast<double*>(p); p += round16(sizeof(double) * (m + 1));
  s.rRloc = reinterpret_cast<double*>(p); p += round16(sizeof(double) * (m + 1));
  s.rLloc = reinterpret_cast<double*>(p); p += round16(sizeof(double) * (m + 1));
  s.piRtot = reinterpret_cast<double*>(p); p += sizeof(double) * 16;
  s.piLtot = reinterpret_cast<double*>(p); p += sizeof(double) * 16;
  s.xch = reinterpret_cast<double*>(p); p += round16(sizeof(double) * 4 * R);
  s.in = reinterpret_cast<double*>(p); p += round16(sizeof(double) * 2 * R);
  s.piR32 = reinterpret_cast<float*>(p); p += round16(sizeof(float) * (m + 1));
  s.piL32 = reinterpret_cast<float*>(p); p += round16(sizeof(float) * (m + 1));
  s.in32 = reinterpret_cast<float*>(p); p += round16(sizeof(float) * 2 * R);
  (void)tsize;
  s.betaR = reinterpret_cast<double*>(p); p += round16(sizeof(double) * m * R);
  s.betaL = reinterpret_cast<double*>(p);
  return s;
}

// byte offset that aligns the dynamic shared-memory window to 128 bytes
__device__ __forceinline__ unsigned smem_align_pad(const void* smem_base) {
  return (128u - ((unsigned)__cvta_generic_to_shared(smem_base) & 127u)) & 127u;
}

// Ratios, prefix products within this CTA, and the per-CTA products of every
// CTA of the cluster (used to fold the incoming partials).
// Products of the separator ratios, by one warp in logarithmic depth (the
// factors are loaded together rather than one dependent load at a time):
//   warp_scan_products: out(j) = f(0) ... f(j) for j < m (inclusive prefix;
//     with `suffix`, out(j) = f(j) ... f(m-1));
//   warp_products: f(0) ... f(m-1), returned in every lane.
// Each lane takes up to 8 consecutive factors (m <= 256).
template <typename Get, typename Put>
__device__ __forceinline__ void warp_scan_products(int m, bool suffix, Get f, Put out) {
  const int lane = threadIdx.x & 31;
  const int K = (m + 31) / 32;
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const int pos = lane * K + k;
    v[k] = (k < K && pos < m) ? f(suffix ? m - 1 - pos : pos) : 1.0;
  }
  double p = 1.0;
#pragma unroll
  for (int k = 0; k < 8; k++) p *= v[k];
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double o = __shfl_up_sync(0xffffffffu, p, d);
    if (lane >= d) p *= o;
  }
  double q = __shfl_up_sync(0xffffffffu, p, 1);
  if (lane == 0) q = 1.0;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const int pos = lane * K + k;
    if (k < K && pos < m) {
      q *= v[k];
      out(suffix ? m - 1 - pos : pos, q);
    }
  }
}
template <typename Get>
__device__ __forceinline__ double warp_products(int m, Get f) {
  const int lane = threadIdx.x & 31;
  double p = 1.0;
  for (int j = lane; j < m; j += 32) p *= f(j);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) p *= __shfl_xor_sync(0xffffffffu, p, o);
  return p;
}

__device__ inline void setup_ratios(const SolveArgs& a, const Smem& s, unsigned c) {
  const int m = a.m, M = a.M, b0 = (int)c * m;
  auto rR = [&](int q) -> double { return (q >= 0 && q <= M + 1) ? a.rR[q] : 0.0; };
  auto rL = [&](int q) -> double { return (q >= 0 && q <= M + 1) ? a.rL[q] : 0.0; };
  const int tid = threadIdx.x;
  for (int j = tid; j <= m; j += blockDim.x) {
    s.rRloc[j] = (j >= 1) ? rR(b0 + j - 1) : 0.0;
    s.rLloc[j] = (j < m) ? rL(b0 + j + 1) : 0.0;
  }
  const int warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (warp == 0) {          // piR_j = rR_{b0} ... rR_{b0+j-1}
    if (tid == 0) { s.piR[0] = 1.0; s.piR32[0] = 1.0f; }
    warp_scan_products(m, false, [&](int j) { return rR(b0 + j); },
                       [&](int j, double p) { s.piR[j + 1] = p; s.piR32[j + 1] = (float)p; });
  } else if (warp == 1) {   // piL_j = rL_{b0+j+1} ... rL_{b0+m}
    if (tid == 32) { s.piL[m] = 1.0; s.piL32[m] = 1.0f; }
    warp_scan_products(m, true, [&](int j) { return rL(b0 + j + 1); },
                       [&](int j, double p) { s.piL[j] = p; s.piL32[j] = (float)p; });
  } else {                  // every CTA's totals, one warp per CTA and direction
    for (int k = warp - 2; k < 2 * a.C; k += nwarps - 2) {
      const int cc = k % a.C, bb = cc * m;
      const double p = k < a.C ? warp_products(m, [&](int j) { return rR(bb + j); })
                               : warp_products(m, [&](int j) { return rL(bb + j + 1); });
      if ((tid & 31) == 0) (k < a.C ? s.piRtot : s.piLtot)[cc] = p;
    }
  }
}

// A4 up to the incoming partials: LR/LL recurrences, exchange, folds.
// pe: the tile's peers (barrier() and ldd(mine, rank): the cluster, or a group
// of a cooperative launch); xbase: where this CTA publishes its partials
// (shared memory, or its scratch block in global memory)
template <typename T, int R, class PE>
__device__ __forceinline__ void separator_partials(const SolveArgs& a, const Smem& s, unsigned c, int parity, PE& pe,
                                                   double* xbase) {
  const int m = a.m;
  const int tid = threadIdx.x;
  const double* betaR = s.betaR;
  const double* betaL = s.betaL;
  double* xch = xbase + parity * 2 * R;
  if (tid < R) {                       // SR, left to right
    const int r = tid;
    double lr = 0.0;
    s.lr[r] = 0.0;
#pragma unroll 2
    for (int j = 1; j <= m; j++) {   // loads do not depend on the chain: only the fma is serial
      lr = fma(s.rRloc[j], lr, betaR[(j - 1) * R + r]);
      s.lr[j * R + r] = lr;
    }
    xch[r] = lr;
  } else if (tid >= 32 && tid < 32 + R) {   // SL, right to left
    const int r = tid - 32;
    double ll = 0.0;
    s.ll[m * R + r] = 0.0;
#pragma unroll 2
    for (int j = m - 1; j >= 0; j--) {
      ll = fma(s.rLloc[j], ll, betaL[j * R + r]);
      s.ll[j * R + r] = ll;
    }
    xch[R + r] = ll;
  }
  pe.barrier();
  // fold the partials of the CTAs to the left (SR) and to the right (SL);
  // remote loads are issued four at a time so that their latencies overlap
  if (tid < R) {
    const int r = tid;
    double in = 0.0;
    for (int c0 = 0; c0 < (int)c; c0 += 4) {
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; k++) v[k] = (c0 + k < (int)c) ? pe.ldd(xch + r, (unsigned)(c0 + k)) : 0.0;
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (c0 + k < (int)c) in = fma(s.piRtot[c0 + k], in, v[k]);
    }
    s.in[r] = in;
    s.in32[r] = tdm_d2f(in);
  } else if (tid >= 32 && tid < 32 + R) {
    const int r = tid - 32;
    double in = 0.0;
    for (int c0 = a.C - 1; c0 > (int)c; c0 -= 4) {
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; k++) v[k] = (c0 - k > (int)c) ? pe.ldd(xch + R + r, (unsigned)(c0 - k)) : 0.0;
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (c0 - k > (int)c) in = fma(s.piLtot[c0 - k], in, v[k]);
    }
    s.in[R + r] = in;
    s.in32[R + r] = tdm_d2f(in);
  }
  __syncthreads();
}

// x(p_{b0+j}) for rhs r, in the solve's type: LR + LL + piR inR + piL inL
template <typename T, int R>
__device__ __forceinline__ T separator_value(const Smem& s, int j, int r) {
  if constexpr (sizeof(T) == 8) {
    return fma(s.piR[j], s.in[r], fma(s.piL[j], s.in[R + r], s.lr[j * R + r] + s.ll[j * R + r]));
  } else {
    const float loc = tdm_d2f(s.lr[j * R + r]) + tdm_d2f(s.ll[j * R + r]);
    return fmaf(s.piR32[j], s.in32[r], fmaf(s.piL32[j], s.in32[R + r], loc));
  }
}

// A2 + A3 over one block held in v[] (overwritten with the forward-eliminated
// values): the two beta dot products and the local sweep's forward pass.
// FULL: all TT rows exist, so no per-row test is compiled in.
template <typename T, int TT, bool FULL>
__device__ __forceinline__ void forward_pass(T (&v)[TT], const T* cf, int nrows, T& bR, T& bL) {
  T g = T(0);
#pragma unroll
  for (int i = 0; i < TT; i++) {
    if (FULL || i < nrows) {
      T gr, gl, lf, unused;
      ld4(cf + i * kNCOEF, gr, gl, lf, unused);
      bR = fma(gr, v[i], bR);
      bL = fma(gl, v[i], bL);
      g = fma(-lf, g, v[i]);
      v[i] = g;
    }
  }
}

// A5 of the plain solve in two parts: the back substitution (independent of
// the separator values, y replaces v), then the correction with the two
// separator values and the store of each row; p points at the block's first
// row of X.
template <typename T, int TT, bool FULL>
__device__ __forceinline__ void backward_y_plain(T (&v)[TT], const T* cf, int nrows) {
  T y = T(0);
#pragma unroll
  for (int i = TT - 1; i >= 0; i--) {
    if (FULL || i < nrows) {
      T cc, invd;
      ld2(cf + i * kNCOEF + kC, cc, invd);
      y = fma(-cc, y, v[i]) * invd;
      v[i] = y;
    }
  }
}
template <typename T, int TT, bool FULL>
__device__ __forceinline__ void correct_store(const T (&v)[TT], const T* cf, int nrows, T xL, T xR, T* p, int64_t ld,
                                              bool col_ok) {
#pragma unroll
  for (int i = 0; i < TT; i++) {
    if (FULL || i < nrows) {
      T phl, phr;
      ld2(cf + i * kNCOEF + kPHIL, phl, phr);
      const T x = fma(phr, xR, fma(phl, xL, v[i]));
      if (col_ok) *p = x;
    }
    p += ld;
  }
}

// A5 of the plain solve: back substitution, correction with the two separator
// values, and the store of each row; p points at the block's first row of X.
template <typename T, int TT, bool FULL>
__device__ __forceinline__ void backward_store(const T (&v)[TT], const T* cf, int nrows, T xL, T xR, T* p,
                                               int64_t ld, bool col_ok) {
  T y = T(0);
  const int last = FULL ? TT - 1 : nrows - 1;
  if (!FULL && last < 0) return;
  p += (int64_t)last * ld;
#pragma unroll
  for (int i = TT - 1; i >= 0; i--) {
    if (FULL || i <= last) {
      T cc, invd, phl, phr;
      ld4(cf + i * kNCOEF + 4, cc, invd, phl, phr);
      y = fma(-cc, y, v[i]) * invd;
      const T x = fma(phr, xR, fma(phl, xL, y));
      if (col_ok) *p = x;
      p -= ld;
    }
  }
}

}  // namespace tdmk
