// tdm_iface_df.cuh -- step A4 (separator values by Theorem 2, eq. theor_2)
// in logarithmic depth: in binary32-pair ("double-float") arithmetic for the
// refined solve (PAIR = true), in binary32 for the plain binary32 solve.
//
// The separator values are x(p_j) = LR_j + LL_j + piR_j in_R + piL_j in_L
// with the two first-order recurrences inside a CTA of m blocks
//     LR_0 = 0,  LR_{j+1} = aR_j LR_j + betaR_j        (left to right)
//     LL_m = 0,  LL_j     = aL_j LL_{j+1} + betaL_j    (right to left)
// and in_R, in_L the partial sums that enter the CTA from the CTAs to its left
// and right.  The multipliers aR_j, aL_j (ratios of neighbouring separators'
// homogeneous solutions, eq. z_vector) depend on the matrix only, so every
// product of them that the evaluation needs is formed once per series, in
// binary64, and kept as pairs:
//   - each recurrence is a Kogge-Stone scan over the 32 lanes of one warp
//     (K = ceil(m / 32) consecutive blocks per lane, scanned sequentially
//     first); level l adds to lane i the value of lane i -/+ 2^l times the
//     product of the multipliers in between;
//   - the partial sums of the other CTAs are folded in one round: every lane
//     takes one CTA's total and multiplies it by the product of the
//     multipliers of the CTAs in between; a shuffle tree adds them up.  The
//     refined solve reads the totals remotely after a cluster barrier
//     (iface_df_fold); the binary32 solve has every CTA push its totals into
//     the others' shared memory, counted by an mbarrier (iface_push_send,
//     iface_push_fold), with no cluster barrier.
// A binary64 chain costs ~60 cycles per step on GB300 and the multipliers of
// an ill-conditioned matrix are close to one, which is why the sums are kept
// in pairs (~2^-46 relative) rather than in binary32.
#pragma once

#include "tdm_df.cuh"
#include "tdm_kernel_common.cuh"
#include "tdm_tma.cuh"

namespace tdmk {

// Shared-memory layout of the A4 arrays for tiles of R right-hand sides and at
// most MM blocks per CTA (byte offsets from the start of the arrays).
struct IfaceOffsets {
  size_t beR, beL;   // float [MM][R+1] beta^R, beta^L of each block (one padding column)
  size_t lr, ll;     // pair [MM+1][R+1] LR_j, LL_j
  size_t aR, aL;     // pair [MM] multipliers
  size_t cpR, cpL;   // pair [MM] aR from the lane start through j; aL from j through the lane end
  size_t ksR, ksL;   // pair [5][32] lane-range products: [i - 2^l + 1, i] and [i, i + 2^l - 1]
  size_t piR, piL;   // pair [MM+1] aR_0 .. aR_{j-1}; aL_j .. aL_{m-1}
  size_t wR, wL;     // pair [16] fold weights of the CTAs to the left / right
  size_t xch;        // pair [2 parity][2 dir][R] this CTA's totals, read by the other CTAs (pairs)
  size_t xin;        // float [2 parity][16 source CTA][R+1] totals pushed by the other CTAs (binary32)
  size_t xbar;       // mbarrier [2 parity] completion of the pushed totals (binary32)
  size_t in;         // pair [2][R] in_R, in_L
  size_t tmp;        // double [96] set-up scratch
  size_t bytes;
};
__host__ __device__ constexpr IfaceOffsets iface_offsets(int R, int MM, bool pair) {
  const size_t es = pair ? 8 : 4;   // LR, LL: pairs, or the leading words only
  IfaceOffsets o{};
  size_t p = 0;
  o.beR = p; p += round16(4 * (size_t)MM * (R + 1));
  o.beL = p; p += round16(4 * (size_t)MM * (R + 1));
  o.lr = p; p += round16(es * (size_t)(MM + 1) * (R + 1));
  o.ll = p; p += round16(es * (size_t)(MM + 1) * (R + 1));
  o.aR = p; p += round16(8 * (size_t)MM);
  o.aL = p; p += round16(8 * (size_t)MM);
  o.cpR = p; p += round16(8 * (size_t)MM);
  o.cpL = p; p += round16(8 * (size_t)MM);
  o.ksR = p; p += 8 * 160;
  o.ksL = p; p += 8 * 160;
  o.piR = p; p += round16(8 * (size_t)(MM + 1));
  o.piL = p; p += round16(8 * (size_t)(MM + 1));
  o.wR = p; p += 8 * 16;
  o.wL = p; p += 8 * 16;
  // pairs: the other CTAs read the totals remotely (xch); binary32: every CTA
  // pushes its totals into the others' xin (see iface_push_send)
  o.xch = p; p += pair ? round16(8 * 4 * (size_t)R) : 0;
  o.xin = p; p += pair ? 0 : round16(4 * 2 * 16 * (size_t)(R + 1));
  o.xbar = p; p += pair ? 0 : 16;
  o.in = p; p += round16(8 * 2 * (size_t)R);
  o.tmp = p; p += 8 * 96;
  o.bytes = p;
  return o;
}

// The arrays at compile-time offsets from `base` (16-byte aligned shared
// memory), so that every access is an immediate offset.
template <int R, int MM, bool PAIR = true>
struct IfaceDF {
  static constexpr IfaceOffsets O = iface_offsets(R, MM, PAIR);
  // Row stride of beR, beL, lr, ll: the scan reads them down a column (lane =
  // block), the blocks write and read them along a row; one padding entry per
  // row keeps both directions free of bank conflicts.
  static constexpr int kRP = R + 1;
  unsigned char* base;
  float2* xg = nullptr;   // the totals in global memory instead (cooperative launches)
  __device__ float* beR() const { return reinterpret_cast<float*>(base + O.beR); }
  __device__ float* beL() const { return reinterpret_cast<float*>(base + O.beL); }
  // LR_j, LL_j entries: pairs (PAIR) or their leading words
  __device__ f2pair ld_lr(int k) const { return ld_entry(O.lr, k); }
  __device__ f2pair ld_ll(int k) const { return ld_entry(O.ll, k); }
  __device__ void st_lr(int k, f2pair v) const { st_entry(O.lr, k, v); }
  __device__ void st_ll(int k, f2pair v) const { st_entry(O.ll, k, v); }
  __device__ f2pair ld_entry(size_t off, int k) const {
    if constexpr (PAIR) {
      const float2 v = reinterpret_cast<const float2*>(base + off)[k];
      return f2pair{v.x, v.y};
    } else {
      return f2pair{reinterpret_cast<const float*>(base + off)[k], 0.f};
    }
  }
  __device__ void st_entry(size_t off, int k, f2pair v) const {
    if constexpr (PAIR) reinterpret_cast<float2*>(base + off)[k] = make_float2(v.h, v.l);
    else reinterpret_cast<float*>(base + off)[k] = v.h;
  }
  __device__ float2* aR() const { return reinterpret_cast<float2*>(base + O.aR); }
  __device__ float2* aL() const { return reinterpret_cast<float2*>(base + O.aL); }
  __device__ float2* cpR() const { return reinterpret_cast<float2*>(base + O.cpR); }
  __device__ float2* cpL() const { return reinterpret_cast<float2*>(base + O.cpL); }
  __device__ float2* ksR() const { return reinterpret_cast<float2*>(base + O.ksR); }
  __device__ float2* ksL() const { return reinterpret_cast<float2*>(base + O.ksL); }
  __device__ float2* piR() const { return reinterpret_cast<float2*>(base + O.piR); }
  __device__ float2* piL() const { return reinterpret_cast<float2*>(base + O.piL); }
  __device__ float2* wR() const { return reinterpret_cast<float2*>(base + O.wR); }
  __device__ float2* wL() const { return reinterpret_cast<float2*>(base + O.wL); }
  __device__ float2* xch() const { return xg ? xg : reinterpret_cast<float2*>(base + O.xch); }
  __device__ float* xin() const { return reinterpret_cast<float*>(base + O.xin); }
  __device__ uint64_t* xbar() const { return reinterpret_cast<uint64_t*>(base + O.xbar); }
  __device__ float2* in() const { return reinterpret_cast<float2*>(base + O.in); }
  __device__ double* tmp() const { return reinterpret_cast<double*>(base + O.tmp); }
};

__device__ __forceinline__ float2 df_of(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ f2pair fp(float2 v) { return f2pair{v.x, v.y}; }
__device__ __forceinline__ float2 f2(f2pair v) { return make_float2(v.h, v.l); }

// a * x + b for pairs, renormalised
__device__ __forceinline__ f2pair df_fma(f2pair a, f2pair x, f2pair b) {
  const float p = a.h * x.h;
  float e = fmaf(a.h, x.h, -p);
  e = fmaf(a.h, x.l, e);
  e = fmaf(a.l, x.h, e);
  const f2pair s = two_sum_f(b.h, p);
  return fast_two_sum_f(s.h, s.l + (e + b.l));
}
__device__ __forceinline__ f2pair df_add(f2pair a, f2pair b) {
  const f2pair s = two_sum_f(a.h, b.h);
  return fast_two_sum_f(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ f2pair shfl_up_pair(f2pair v, int d) {
  return f2pair{__shfl_up_sync(0xffffffffu, v.h, d), __shfl_up_sync(0xffffffffu, v.l, d)};
}
__device__ __forceinline__ f2pair shfl_down_pair(f2pair v, int d) {
  return f2pair{__shfl_down_sync(0xffffffffu, v.h, d), __shfl_down_sync(0xffffffffu, v.l, d)};
}
__device__ __forceinline__ f2pair shfl_xor_pair(f2pair v, int d) {
  return f2pair{__shfl_xor_sync(0xffffffffu, v.h, d), __shfl_xor_sync(0xffffffffu, v.l, d)};
}
// The scan, fold and separator evaluation below run in pairs (PAIR = true,
// ~2^-46 relative) or in plain binary32 on the leading words (PAIR = false:
// the products are the same, the sums are rounded to binary32 at every step).
template <bool PAIR>
__device__ __forceinline__ f2pair mfma(f2pair a, f2pair x, f2pair b) {
  if constexpr (PAIR) return df_fma(a, x, b);
  else return f2pair{fmaf(a.h, x.h, b.h), 0.f};
}
template <bool PAIR>
__device__ __forceinline__ f2pair madd(f2pair a, f2pair b) {
  if constexpr (PAIR) return df_add(a, b);
  else return f2pair{a.h + b.h, 0.f};
}
template <bool PAIR>
__device__ __forceinline__ f2pair mshfl_up(f2pair v, int d) {
  if constexpr (PAIR) return shfl_up_pair(v, d);
  else return f2pair{__shfl_up_sync(0xffffffffu, v.h, d), 0.f};
}
template <bool PAIR>
__device__ __forceinline__ f2pair mshfl_down(f2pair v, int d) {
  if constexpr (PAIR) return shfl_down_pair(v, d);
  else return f2pair{__shfl_down_sync(0xffffffffu, v.h, d), 0.f};
}
template <bool PAIR>
__device__ __forceinline__ f2pair mshfl_xor(f2pair v, int d) {
  if constexpr (PAIR) return shfl_xor_pair(v, d);
  else return f2pair{__shfl_xor_sync(0xffffffffu, v.h, d), 0.f};
}
template <bool PAIR>
__device__ __forceinline__ f2pair mld(const float2* p) {
  if constexpr (PAIR) return fp(*p);
  else return f2pair{*reinterpret_cast<const float*>(p), 0.f};
}

__device__ __forceinline__ float2 ld_cluster_f32x2(const float2* local, unsigned rank) {
  const unsigned laddr = (unsigned)__cvta_generic_to_shared(local);
  unsigned raddr;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(raddr) : "memory");
  return v;
}

// Per-series set-up of every product (binary64, then pairs).  All threads of
// the CTA call it; it synchronizes the CTA.  rR, rL have M + 2 entries; the
// multipliers of CTA c are aR_j = rR[c m + j], aL_j = rL[c m + j + 1].
template <int R, int MM, bool PAIR>
__device__ __forceinline__ void iface_df_setup(const IfaceDF<R, MM, PAIR>& f, const double* rR, const double* rL, int M,
                                               int m, int C, unsigned c) {
  const int tid = threadIdx.x, nt = blockDim.x;
  auto gR = [&](int q) -> double { return (q >= 0 && q <= M + 1) ? rR[q] : 0.0; };
  auto gL = [&](int q) -> double { return (q >= 0 && q <= M + 1) ? rL[q] : 0.0; };
  const int K = (m + 31) / 32, nl = (m + K - 1) / K;
  const int b0 = (int)c * m;
  double* AR = f.tmp();        // [32] lane products
  double* AL = f.tmp() + 32;
  double* TR = f.tmp() + 64;   // [16] CTA totals
  double* TL = f.tmp() + 80;
  for (int u = tid; u < 64; u += nt) {
    {               // one lane of one direction: multipliers, in-lane products, lane product
      const int lane = u & 31;
      double p = 1.0;
      if (lane < nl) {
        const int j0 = lane * K, j1 = min(j0 + K, m);
        if (u < 32) {
          for (int j = j0; j < j1; j++) { const double a = gR(b0 + j); f.aR()[j] = df_of(a); p *= a; f.cpR()[j] = df_of(p); }
        } else {
          for (int j = j1 - 1; j >= j0; j--) { const double a = gL(b0 + j + 1); f.aL()[j] = df_of(a); p *= a; f.cpL()[j] = df_of(p); }
        }
      }
      (u < 32 ? AR : AL)[lane] = p;
    }
  }
  // prefix products from the left and from the right, and the totals of every
  // CTA of the cluster (one warp per CTA and direction); each warp loads its
  // factors together and multiplies in logarithmic depth
  const int warp = tid >> 5, nwarps = nt >> 5;
  if (warp == 0) {
    if (tid == 0) f.piR()[0] = df_of(1.0);
    warp_scan_products(m, false, [&](int j) { return gR(b0 + j); }, [&](int j, double p) { f.piR()[j + 1] = df_of(p); });
  } else if (warp == 1) {
    if (tid == 32) f.piL()[m] = df_of(1.0);
    warp_scan_products(m, true, [&](int j) { return gL(b0 + j + 1); }, [&](int j, double p) { f.piL()[j] = df_of(p); });
  } else {
    for (int k = warp - 2; k < 2 * C; k += nwarps - 2) {
      const int cc = k % C;
      const double p = k < C ? warp_products(m, [&](int j) { return gR(cc * m + j); })
                             : warp_products(m, [&](int j) { return gL(cc * m + j + 1); });
      if ((tid & 31) == 0) (k < C ? TR : TL)[cc] = p;
    }
  }
  __syncthreads();
  for (int u = tid; u < 320 + 32; u += nt) {
    if (u < 320) {   // scan-level products
      const bool left = u < 160;
      const int l = (u % 160) / 32, lane = u % 32, d = 1 << l;
      double p = 1.0;
      if (left) {
        for (int q = lane - d + 1; q <= lane; q++) if (q >= 0) p *= AR[q];
        f.ksR()[l * 32 + lane] = df_of(p);
      } else {
        for (int q = lane; q <= lane + d - 1; q++) if (q < 32) p *= AL[q];
        f.ksL()[l * 32 + lane] = df_of(p);
      }
    } else {         // fold weights
      const int k = u - 320, cc = k % 16;
      double p = 0.0;
      if (k < 16) {
        if (cc < (int)c) { p = 1.0; for (int q = cc + 1; q < (int)c; q++) p *= TR[q]; }
        f.wR()[cc] = df_of(p);
      } else {
        if (cc > (int)c && cc < C) { p = 1.0; for (int q = (int)c + 1; q < cc; q++) p *= TL[q]; }
        f.wL()[cc] = df_of(p);
      }
    }
  }
  __syncthreads();
}

// LR_j, LL_j of this CTA and its totals (into xch[parity]); one warp scans a
// column in both directions.  The betas must be visible (CTA barrier).
// AP: the arithmetic of the scan -- pairs, or binary32 on the leading words of
// the same storage (a correction solve of the refined path needs only binary32
// separator values).
template <int R, int MM, bool PAIR = true, bool AP = PAIR>
__device__ __forceinline__ void iface_df_scan(const IfaceDF<R, MM, PAIR>& f, int m, int parity) {
  constexpr int RP = IfaceDF<R, MM, PAIR>::kRP;
  constexpr int KMAX = (MM + 31) / 32;   // most blocks per lane (1: every lane holds one block)
  const int lane = threadIdx.x & 31;
  const int K = KMAX == 1 ? 1 : (m + 31) / 32, nl = (m + K - 1) / K;
  const int j0 = lane * K, j1 = min(j0 + K, m);
  for (int r = threadIdx.x >> 5; r < R; r += blockDim.x >> 5) {
    // in-lane sequential parts (stored, then completed with what enters the lane)
    f2pair accR{0.f, 0.f}, accL{0.f, 0.f};
    for (int j = j0; j < j1; j++) {
      accR = mfma<AP>(mld<AP>(&f.aR()[j]), accR, f2pair{f.beR()[j * RP + r], 0.f});
      if (KMAX > 1 && K > 1) f.st_lr((j + 1) * RP + r, accR);
    }
    for (int j = j1 - 1; j >= j0; j--) {
      accL = mfma<AP>(mld<AP>(&f.aL()[j]), accL, f2pair{f.beL()[j * RP + r], 0.f});
      if (KMAX > 1 && K > 1) f.st_ll(j * RP + r, accL);
    }
#pragma unroll
    for (int l = 0; l < 5; l++) {
      const int d = 1 << l;
      const f2pair pR = mshfl_up<AP>(accR, d);
      const f2pair pL = mshfl_down<AP>(accL, d);
      if (lane >= d && lane < nl) accR = mfma<AP>(mld<AP>(&f.ksR()[l * 32 + lane]), pR, accR);
      if (lane + d < nl) accL = mfma<AP>(mld<AP>(&f.ksL()[l * 32 + lane]), pL, accL);
    }
    if (KMAX > 1 && K > 1) {
      f2pair eR = mshfl_up<AP>(accR, 1);     // everything left of this lane
      f2pair eL = mshfl_down<AP>(accL, 1);   // everything right of it
      if (lane == 0) eR = f2pair{0.f, 0.f};
      if (lane + 1 >= nl) eL = f2pair{0.f, 0.f};
      for (int j = j0; j < j1; j++) {
        f.st_lr((j + 1) * RP + r, mfma<AP>(mld<AP>(&f.cpR()[j]), eR, f.ld_lr((j + 1) * RP + r)));
        f.st_ll(j * RP + r, mfma<AP>(mld<AP>(&f.cpL()[j]), eL, f.ld_ll(j * RP + r)));
      }
    } else if (j0 < m) {   // one block per lane: the scan already holds the values
      f.st_lr((j0 + 1) * RP + r, accR);
      f.st_ll(j0 * RP + r, accL);
    }
    if (lane == 0) {
      f.st_lr(r, f2pair{0.f, 0.f});
      f.st_ll(m * RP + r, f2pair{0.f, 0.f});
    }
    __syncwarp();
    if constexpr (PAIR) {
      if (lane == 0) {
        f.xch()[(parity * 2 + 0) * R + r] = f2(f.ld_lr(m * RP + r));
        f.xch()[(parity * 2 + 1) * R + r] = f2(f.ld_ll(r));
      }
    }
  }
}

// binary32: this CTA's totals of every column pushed into the other CTAs'
// shared memory (after iface_df_scan, by the same warps): CTA cc receives
// LR_m when it lies to the right, LL_0 when it lies to the left, at
// xin[parity][c][r], and its barrier xbar[parity] counts the bytes.  No
// memory fence is needed: the store carries its own completion.
__device__ __forceinline__ void st_async_cluster_f32(float* local_dst, unsigned rank, float v, uint64_t* local_bar) {
  const unsigned ldst = (unsigned)__cvta_generic_to_shared(local_dst);
  const unsigned lbar = (unsigned)__cvta_generic_to_shared(local_bar);
  unsigned rdst, rbar;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rdst) : "r"(ldst), "r"(rank));
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbar) : "r"(lbar), "r"(rank));
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(rdst), "r"(__float_as_uint(v)), "r"(rbar) : "memory");
}
template <int R, int MM>
__device__ __forceinline__ void iface_push_send(const IfaceDF<R, MM, false>& f, int m, int C, unsigned c, int parity) {
  constexpr int RP = IfaceDF<R, MM, false>::kRP;
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < R; r += blockDim.x >> 5) {
    if (lane < C && lane != (int)c) {
      const float v = lane > (int)c ? f.ld_lr(m * RP + r).h : f.ld_ll(r).h;
      st_async_cluster_f32(f.xin() + (parity * 16 + (int)c) * (R + 1) + r, (unsigned)lane, v, f.xbar() + parity);
    }
  }
}
// bytes that arrive at xbar[parity] per tile
template <int R>
__host__ __device__ constexpr uint32_t iface_push_bytes(int C) { return (uint32_t)((C - 1) * R * 4); }

// binary32 fold of the pushed totals (after xbar[parity] completed): one warp
// per column, lanes 0-15 for the CTAs to the left, 16-31 for those to the
// right, all reads local.
template <int R, int MM>
__device__ __forceinline__ void iface_push_fold(const IfaceDF<R, MM, false>& f, int C, unsigned c, int parity) {
  const int lane = threadIdx.x & 31, cc = lane & 15;
  const bool left = lane < 16;
  const bool valid = left ? (cc < (int)c) : (cc > (int)c && cc < C);
  const float w = valid ? (left ? f.wR()[cc].x : f.wL()[cc].x) : 0.f;
  const float* src = f.xin() + (parity * 16 + cc) * (R + 1);
  for (int r = threadIdx.x >> 5; r < R; r += blockDim.x >> 5) {
    float v = valid ? w * src[r] : 0.f;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) f.in()[r] = make_float2(v, 0.f);
    if (lane == 16) f.in()[R + r] = make_float2(v, 0.f);
  }
}

// The cluster's CTAs as the peers of a tile: loads from the same
// shared-memory offset in another CTA.
struct ClusterPeers {
  __device__ float2 ld2(const float2* mine, unsigned rank) const { return ld_cluster_f32x2(mine, rank); }
};

// The peers of a tile and their barrier.
//  * Cluster (COOP false): the CTAs of the thread-block cluster.  Barriers are
//    the hardware cluster barrier; what the peers read sits in shared memory
//    and is read through the cluster's shared-memory window.
//  * Group (COOP true): g consecutive CTAs of a cooperative launch (every CTA
//    of the grid resident at once).  A barrier is a counter in global memory:
//    each CTA, after its writes and a CTA barrier, adds 1 from one thread with
//    release semantics (the barrier orders the other threads' writes before
//    it), and waits
//    until the count reaches its own arrivals times g (a bounded spin by one
//    thread; on time-out it records kDevErrGroupTimeout and stops waiting).
//    What the peers read sits in a scratch block of kScr floats per CTA in
//    global memory, read with gpu-scope loads (not through L1) after the
//    barrier.  Ranks are group-relative: rank k is the CTA first + k.
constexpr int kGroupSpinLimit = 1 << 21;
template <bool COOP>
struct Link {
  unsigned me = 0;         // this CTA's index in the grid (COOP)
  unsigned first = 0;      // the grid index of the group's rank 0 (COOP)
  int stride = 0;          // floats between consecutive CTAs' scratch blocks (COOP)
  unsigned g = 0;          // CTAs of the group (COOP)
  unsigned* ctr = nullptr; // the group's counter (COOP)
  int* err = nullptr;
  unsigned narr = 0;       // this CTA's arrivals so far
  bool broken = false;     // a wait timed out (thread 0)
  int spin_limit = kGroupSpinLimit;   // polls before a wait gives up
  __device__ const float* at(const float* mine, unsigned rank) const {
    return mine + ((int)(first + rank) - (int)me) * stride;
  }
  __device__ float ld(const float* mine, unsigned rank) const {
    if constexpr (COOP) {
      float v;
      asm volatile("ld.relaxed.gpu.f32 %0, [%1];" : "=f"(v) : "l"(at(mine, rank)) : "memory");
      return v;
    } else {
      return ld_cluster_f32(mine, rank);
    }
  }
  __device__ double ldd(const double* mine, unsigned rank) const {
    if constexpr (COOP) {
      const double* p = reinterpret_cast<const double*>(at(reinterpret_cast<const float*>(mine), rank));
      double v;
      asm volatile("ld.relaxed.gpu.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
      return v;
    } else {
      return ld_cluster_f64(mine, rank);
    }
  }
  __device__ float2 ld2(const float2* mine, unsigned rank) const {
    if constexpr (COOP) {
      const float* p = at(reinterpret_cast<const float*>(mine), rank);
      float2 v;
      asm volatile("ld.relaxed.gpu.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
      return v;
    } else {
      return ld_cluster_f32x2(mine, rank);
    }
  }
  __device__ void arrive() {
    if constexpr (COOP) {
      __syncthreads();
      if (g == 1) return;   // no peer: the CTA barrier orders its own scratch
      if (threadIdx.x == 0) {   // the CTA barrier orders the other threads' writes before this release
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
      }
      narr++;
    } else {
      cluster_arrive();
    }
  }
  __device__ void wait() {
    if constexpr (COOP) {
      if (g == 1) {
        __syncthreads();
        return;
      }
      if (threadIdx.x == 0 && !broken) {
        const unsigned target = narr * g;
        for (int it = 0;; it++) {
          unsigned v;
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
          if (v >= target) break;
          if (it >= spin_limit) {
            broken = true;
            atomicExch(err, kDevErrGroupTimeout);
            break;
          }
          if (it >= 32) __nanosleep(64);
        }
      }
      __syncthreads();
    } else {
      cluster_wait();
    }
  }
  __device__ void barrier() {
    if constexpr (COOP) {
      arrive();
      wait();
    } else {
      cluster_barrier();
    }
  }
};

// in_R, in_L of every column from the other CTAs' totals (after the barrier
// that published them): one warp per column, lanes 0-15 for the CTAs to the
// left, 16-31 for those to the right.  The C CTAs that share the tile are
// ranks base .. base + C - 1 of the peers `pe` (a cluster, or a group of a
// cooperative launch); c is this CTA's place among them.
template <int R, int MM, bool PAIR = true, bool AP = PAIR, class P = ClusterPeers>
__device__ __forceinline__ void iface_df_fold(const IfaceDF<R, MM, PAIR>& f, int C, unsigned c, int parity,
                                              unsigned base = 0, const P& pe = P{}) {
  const int lane = threadIdx.x & 31, cc = lane & 15;
  const bool left = lane < 16;
  const bool valid = left ? (cc < (int)c) : (cc > (int)c && cc < C);
  for (int r = threadIdx.x >> 5; r < R; r += blockDim.x >> 5) {
    f2pair v{0.f, 0.f};
    if (valid) {
      const float2 x = pe.ld2(f.xch() + (parity * 2 + (left ? 0 : 1)) * R + r, base + (unsigned)cc);
      v = mfma<AP>(mld<AP>(left ? &f.wR()[cc] : &f.wL()[cc]), fp(x), f2pair{0.f, 0.f});
    }
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v = madd<AP>(v, mshfl_xor<AP>(v, o));
    if (lane == 0) f.in()[r] = f2(v);
    if (lane == 16) f.in()[R + r] = f2(v);
  }
}

// x(p_j) for column r, as a pair (AP) or a binary32 value in .h
template <int R, int MM, bool PAIR = true, bool AP = PAIR>
__device__ __forceinline__ f2pair iface_df_sep_pair(const IfaceDF<R, MM, PAIR>& f, int j, int r) {
  constexpr int RP = IfaceDF<R, MM, PAIR>::kRP;
  f2pair x = madd<AP>(f.ld_lr(j * RP + r), f.ld_ll(j * RP + r));
  x = mfma<AP>(mld<AP>(&f.piR()[j]), mld<AP>(&f.in()[r]), x);
  x = mfma<AP>(mld<AP>(&f.piL()[j]), mld<AP>(&f.in()[R + r]), x);
  return x;
}
// x(p_j) for column r, rounded to binary32
template <int R, int MM, bool PAIR = true, bool AP = PAIR>
__device__ __forceinline__ float iface_df_sep(const IfaceDF<R, MM, PAIR>& f, int j, int r) {
  const f2pair x = iface_df_sep_pair<R, MM, PAIR, AP>(f, j, r);
  return x.h + x.l;
}

}  // namespace tdmk
