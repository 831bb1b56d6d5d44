// tdm_solve.cu -- step 2 of Algorithms 3/4 (Sections 3.3-3.4): the per
// right-hand-side solve, fused into one persistent kernel per precision.
//
// Work decomposition.  A thread-block cluster owns a tile of R right-hand
// sides and ALL n rows; CTA c of the cluster owns m consecutive blocks of t
// rows (the paper's PE owns one sub-vector, Section 2); thread (block bl,
// rhs r) owns the t rows of one block for one right-hand side, so a warp's
// lanes touch consecutive right-hand sides of the same row.
//
// Per tile:
//  load  the CTA's rows of the tile arrive in shared memory by TMA (issued
//        while the previous tile was being computed) and move to registers;
//  A2    beta^R_b = sum_{i in block b} G_{p_{b+1}}(i) F_i,
//        beta^L_b = sum_{i in block b} G_{p_b}(i) F_i            (eq. beta_symn)
//  A3    forward elimination of the block interior's local sweep (Lemma 1),
//        fused with A2 in one pass over the rows held in registers;
//  A4    separator values by Theorem 2 (eq. theor_2).  With the ratios
//        rR_q = Z^R_{p_q}(p_{q+1}) and rL_q = Z^L_{p_q}(p_{q-1}) the two sums of
//        Theorem 2 obey first-order recurrences
//            SR_q = beta^R_{q-1} + rR_{q-1} SR_{q-1},
//            SL_q = beta^L_q     + rL_{q+1} SL_{q+1},    x(p_q) = SR_q + SL_q,
//        because Z^R_{p_j}(p_i) = prod_{k=j}^{i-1} rR_k (a homogeneous solution
//        restricted to [p_k, n) is a multiple of Z^R_{p_k}), and likewise for
//        Z^L.  Each CTA runs both recurrences over its own blocks from zero
//        (LR, LL): sequentially in binary64 for the binary64 solve, as warp
//        scans in binary32 (tdm_iface_df.cuh) for the binary32 solve; the CTAs
//        exchange one partial per direction through distributed shared memory
//        (binary64: remote loads after a cluster barrier; binary32: pushed with
//        st.async and counted by an mbarrier); the incoming partials inR, inL
//        enter as x(p_q) = LR_q + LL_q + piR_q inR + piL_q inL with prefix
//        products piR, piL of the ratios.  This is the GPU form of the
//        dichotomy's level-by-level schedule (Algorithm 4): O(M) work.
//  A5    back substitution of the local sweep and the correction
//        x_i = y_i + phiL_i x(p_b) + phiR_i x(p_{b+1}); one coalesced store.
// F is read once and X written once per tile.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "tdm_internal.cuh"
#include "tdm_tma.cuh"

bool tdm_encode_tma_2d(CUtensorMap* out, const void* base, bool fp64, uint64_t cols, uint64_t rows,
                       uint64_t ld_bytes, uint32_t box_cols, uint32_t box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  });
  const uint64_t es = fp64 ? 8 : 4;
  if (!fn || (reinterpret_cast<uintptr_t>(base) % 16) || (ld_bytes % 16) || ((box_cols * es) % 16) ||
      box_cols > 256 || box_rows > 256 || cols < box_cols || ld_bytes >= (1ull << 40))
    return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld_bytes};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(out, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

#include "tdm_kernel_common.cuh"
#include "tdm_iface_df.cuh"

namespace {
using namespace tdmk;

// COOP (binary64 only): a cooperative launch without clusters; groups of a.C
// consecutive CTAs exchange their partials through a.scr and a counter per
// group (Link), where clusters of a.C CTAs would leave many SMs idle.
template <typename T, int R, int TT, int MAXT, bool TMA, bool COOP = false>
__global__ void __launch_bounds__(MAXT, (sizeof(T) == 4 ? 2 : 1)) k_solve(const __grid_constant__ CUtensorMap tmF, const SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int wait_ok;
  unsigned char* base = smem_raw + smem_align_pad(smem_raw);
  T* fbuf = reinterpret_cast<T*>(base);
  T* scf = reinterpret_cast<T*>(base + fbuf_bytes(a.m, TT, R, (int)sizeof(T), TMA));   // [m*t][8]
  // A4 state: binary64 recurrences for the binary64 solve; for the binary32
  // solve, binary32 scans over the same precomputed products as the refined
  // kernel (its separator values only need binary32 accuracy)
  unsigned char* const a4 = reinterpret_cast<unsigned char*>(scf) + coef_bytes(a.m, TT, (int)sizeof(T));
  const Smem s = carve(a4, a.m, R, (int)sizeof(T));
  constexpr int MM = MAXT / R;
  const IfaceDF<R, MM, false> f{a4};
  static_assert(!COOP || sizeof(T) == 8, "the cooperative form is the binary64 solve's");
  const unsigned c = COOP ? blockIdx.x % a.C : cluster_rank();
  const int tid = threadIdx.x;
  const int r = tid % R;
  const int bl = tid / R;
  const int b = (int)c * a.m + bl;
  const bool blk_ok = (bl < a.m) && (b < a.M);
  const int64_t row0 = (int64_t)b * TT;
  // rows of this thread's block that exist (0 for padding threads)
  const int nrows = blk_ok ? (int)((a.n - row0) < TT ? (a.n - row0) : TT) : 0;
  const int rows_cta = a.m * TT;
  const int64_t cta_row0 = (int64_t)c * rows_cta;
  const T* __restrict__ F = static_cast<const T*>(a.F);
  T* __restrict__ X = static_cast<T*>(a.X);
  const T* __restrict__ coef = static_cast<const T*>(a.coef);
  const int n = a.n;

  if constexpr (sizeof(T) == 8) setup_ratios(a, s, c);
  else iface_df_setup(f, a.rR, a.rL, a.M, a.m, a.C, c);
  {   // this CTA's coefficient rows stay in shared memory for every tile
    const int nvec = rows_cta * kNCOEF / 4;
    for (int k = tid; k < nvec; k += blockDim.x) {
      const int64_t row = cta_row0 + (k * 4) / kNCOEF;
      T x = T(0), y = T(0), z = T(0), w = T(0);
      if (row < n) ld4(coef + cta_row0 * kNCOEF + (int64_t)k * 4, x, y, z, w);
      T* d = scf + (size_t)k * 4 + (size_t)((k * 4) / (TT * kNCOEF)) * kCPAD;
      d[0] = x; d[1] = y; d[2] = z; d[3] = w;
    }
  }
  if (TMA && tid == 0) tdm_mbar_init(&mbar, 1);
  if constexpr (sizeof(T) == 4) {
    if (tid == 0) {
      tdm_mbar_init(f.xbar() + 0, 1);
      tdm_mbar_init(f.xbar() + 1, 1);
    }
    // every CTA's exchange barriers exist before any CTA pushes to them
    cluster_barrier();
  } else {
    __syncthreads();
  }

  const int cluster_id = blockIdx.x / a.C;
  const int nclusters = gridDim.x / a.C;
  Link<COOP> lk;
  double* xbase = nullptr;
  if constexpr (sizeof(T) == 8) xbase = COOP ? a.scr + (size_t)blockIdx.x * 4 * R : s.xch;
  if constexpr (COOP) {
    lk.me = blockIdx.x;
    lk.first = (unsigned)(cluster_id * a.C);
    lk.stride = 8 * R;   // floats: 4R doubles per CTA
    lk.g = (unsigned)a.C;
    lk.ctr = a.ctr + 32 * cluster_id;
    lk.err = a.err;
  }
  const uint32_t tile_bytes = (uint32_t)rows_cta * R * sizeof(T);
  const int nbox = rows_cta / a.box_rows;
  auto issue = [&](int tile) {
    tdm_mbar_expect_tx(&mbar, tile_bytes);
    for (int k = 0; k < nbox; k++)
      tdm_tma_load_2d(fbuf + (size_t)k * a.box_rows * R, &tmF, tile * R, (int)(cta_row0 + (int64_t)k * a.box_rows), &mbar);
  };
  if (TMA && tid == 0 && cluster_id < a.ntiles) issue(cluster_id);

  uint32_t phase = 0;
  uint32_t xphase = 0;   // bit p: phase of xbar[p]
  bool abort = false;
  int parity = 0;
  for (int tile = cluster_id; tile < a.ntiles; tile += nclusters) {
    const int64_t col = (int64_t)tile * R + r;
    const bool col_ok = col < a.N;
    if constexpr (sizeof(T) == 4) {
      if (tid == 0) tdm_mbar_expect_tx(f.xbar() + parity, iface_push_bytes<R>(a.C));
    }
    T v[TT];
    if constexpr (TMA) {
      if (!abort && !tdm_mbar_wait_cta(&mbar, phase, a.err, &wait_ok)) abort = true;
      phase ^= 1u;
      // rows beyond n arrive as zeros (TMA fills out-of-bounds elements with zero)
      const T* src = fbuf + (size_t)bl * TT * R + r;
#pragma unroll
      for (int i = 0; i < TT; i++) v[i] = blk_ok ? src[i * R] : T(0);
      __syncthreads();
      if (tid == 0 && !abort && tile + nclusters < a.ntiles) {
        tdm_fence_proxy_async();
        issue(tile + nclusters);
      }
    } else {
      const T* Fp = F + row0 * a.ldF + col;
#pragma unroll
      for (int i = 0; i < TT; i++) v[i] = (i < nrows && col_ok) ? Fp[(int64_t)i * a.ldF] : T(0);
    }
    // A2 + A3 forward: one pass over the rows
    const T* cfb = scf + (size_t)bl * (TT * kNCOEF + kCPAD);
    T bR = T(0), bL = T(0);
    if (nrows == TT) forward_pass<T, TT, true>(v, cfb, nrows, bR, bL);
    else forward_pass<T, TT, false>(v, cfb, nrows, bR, bL);
    T xL = T(0), xR = T(0);
    if constexpr (sizeof(T) == 8) {
      if (bl < a.m) {
        s.betaR[bl * R + r] = bR;
        s.betaL[bl * R + r] = bL;
      }
      __syncthreads();
      separator_partials<T, R>(a, s, c, parity, lk, xbase);
      if (blk_ok) {
        if (b >= 1) xL = separator_value<T, R>(s, bl, r);
        if (b + 1 <= a.M - 1) xR = separator_value<T, R>(s, bl + 1, r);
      }
    } else {
      if (bl < a.m) {
        f.beR()[bl * f.kRP + r] = bR;
        f.beL()[bl * f.kRP + r] = bL;
      }
      __syncthreads();
      iface_df_scan<R, MM, false>(f, a.m, parity);
      iface_push_send<R, MM>(f, a.m, a.C, c, parity);
      // the back substitution overlaps the exchange of the CTA totals
      if (nrows == TT) backward_y_plain<T, TT, true>(v, cfb, nrows);
      else backward_y_plain<T, TT, false>(v, cfb, nrows);
      if (!abort && !tdm_mbar_wait(f.xbar() + parity, (xphase >> parity) & 1u, a.err)) abort = true;
      xphase ^= 1u << parity;
      iface_push_fold<R, MM>(f, a.C, c, parity);
      __syncthreads();
      if (blk_ok) {
        if (b >= 1) xL = iface_df_sep<R, MM, false>(f, bl, r);
        if (b + 1 <= a.M - 1) xR = iface_df_sep<R, MM, false>(f, bl + 1, r);
      }
      T* Xp = X + row0 * a.ldX + col;
      if (nrows == TT) correct_store<T, TT, true>(v, cfb, nrows, xL, xR, Xp, a.ldX, col_ok);
      else correct_store<T, TT, false>(v, cfb, nrows, xL, xR, Xp, a.ldX, col_ok);
      parity ^= 1;
      continue;
    }
    // A5: back substitution + correction + store
    T* Xp = X + row0 * a.ldX + col;
    if (nrows == TT) backward_store<T, TT, true>(v, cfb, nrows, xL, xR, Xp, a.ldX, col_ok);
    else backward_store<T, TT, false>(v, cfb, nrows, xL, xR, Xp, a.ldX, col_ok);
    parity ^= 1;
  }
  // no CTA may leave while a peer can still read its shared memory (the
  // cooperative form's scratch stays readable)
  if constexpr (!COOP) cluster_barrier();
}

// ---------------------------------------------------------------------------
// launch configuration
// ---------------------------------------------------------------------------
struct Cfg {
  int R = 0, m = 0, C = 0, threads = 0, box_rows = 0;
  bool tma = false;
  size_t smem = 0;
};

// binary32: 512 threads and at most ~111 KB of shared memory, so that two CTAs
// (of different clusters) share an SM and one's exchange phase overlaps the
// other's loads; binary64: 512 threads with 32 doubles per thread in registers.
bool choose_cfg(int M, int t, bool fp64, Cfg& cfg) {
  const int maxt = 512;
  const int pref = fp64 ? 16 : 32;   // the widest tile that fits; narrower ones for larger n
  for (int R = pref; R >= 8; R /= 2) {
    if (R != 8 && R != 16 && R != 32) continue;
    const int m_max = maxt / R;
    const int C = (M + m_max - 1) / m_max;
    if (C > 16) continue;
    const int m = (M + C - 1) / C;
    int threads = ((m * R + 31) / 32) * 32;
    if (threads < 96) threads = 96;
    cfg.R = R; cfg.m = m; cfg.C = C; cfg.threads = threads;
    int g = 1;
    for (int d = 1; d <= m; d++)
      if (m % d == 0 && d * t <= 256) g = d;
    cfg.box_rows = g * t;
    return true;
  }
  return false;
}

template <typename T, int R, int TT, int MAXT, bool TMA>
tdm_status launch_t(const CUtensorMap& map, const SolveArgs& args, const Cfg& cfg, cudaStream_t s) {
  auto kern = k_solve<T, R, TT, MAXT, TMA>;
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t, int>, int> occ;  // (device, C, smem, threads) -> clusters
  int dev = 0;
  cudaGetDevice(&dev);
  TDM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem));
  if (cfg.C > 8) TDM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cfg.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(cfg.threads);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  int maxc = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(dev, cfg.C, cfg.smem, cfg.threads);
    auto it = occ.find(key);
    if (it != occ.end()) {
      maxc = it->second;
    } else {
      lc.gridDim = dim3(cfg.C);
      if (cudaOccupancyMaxActiveClusters(&maxc, (void*)kern, &lc) != cudaSuccess || maxc < 1) {
        (void)cudaGetLastError();
        maxc = 1;
      }
      occ[key] = maxc;
    }
  }
  const int nclusters = args.ntiles < maxc ? args.ntiles : maxc;
  lc.gridDim = dim3(nclusters * cfg.C);
  TDM_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, map, args));
  return TDM_OK;
}

// The cooperative binary64 solve: CTAs per SM of its kernel, and the launch
// (whole groups of cfg.C CTAs, at most the plan's scratch; the groups'
// counters are zeroed on the stream first).
template <int R, int TT, bool TMA>
int coop_blocks(const Cfg& cfg) {
  auto kern = k_solve<double, R, TT, 512, TMA, true>;
  int dev = 0, sms = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, cfg.threads, cfg.smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return nb * sms;
}
template <int R, int TT, bool TMA>
tdm_status launch_coop_t(const CUtensorMap& map, const SolveArgs& args, const Cfg& cfg, int max_grid, cudaStream_t s) {
  auto kern = k_solve<double, R, TT, 512, TMA, true>;
  const int blocks = std::min(coop_blocks<R, TT, TMA>(cfg), max_grid);
  const int groups = std::min(blocks / cfg.C, args.ntiles);
  if (groups < 1) return TDM_ERR_NOT_IMPLEMENTED;
  TDM_CUDA_TRY(cudaMemsetAsync(args.ctr, 0, sizeof(unsigned) * 32 * groups, s));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.gridDim = dim3(groups * cfg.C);
  lc.blockDim = dim3(cfg.threads);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  TDM_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, map, args));
  return TDM_OK;
}
template <int TT>
tdm_status dispatch_coop(const CUtensorMap& map, const SolveArgs& args, const Cfg& cfg, int max_grid, cudaStream_t s) {
  switch (cfg.R * 2 + (cfg.tma ? 1 : 0)) {
    case 8 * 2 + 1: return launch_coop_t<8, TT, true>(map, args, cfg, max_grid, s);
    case 16 * 2 + 1: return launch_coop_t<16, TT, true>(map, args, cfg, max_grid, s);
    case 8 * 2: return launch_coop_t<8, TT, false>(map, args, cfg, max_grid, s);
    case 16 * 2: return launch_coop_t<16, TT, false>(map, args, cfg, max_grid, s);
  }
  return TDM_ERR_NOT_IMPLEMENTED;
}
// CTAs that clusters of the cluster form (cfg.C CTAs each) hold at once
template <int R, int TT, bool TMA>
int cluster_slots(const Cfg& cfg) {
  auto kern = k_solve<double, R, TT, 512, TMA, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem) != cudaSuccess ||
      (cfg.C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cfg.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(cfg.threads);
  lc.dynamicSmemBytes = cfg.smem;
  lc.attrs = at;
  lc.numAttrs = 1;
  lc.gridDim = dim3(cfg.C);
  int maxc = 0;
  if (cudaOccupancyMaxActiveClusters(&maxc, (void*)kern, &lc) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return maxc * cfg.C;
}

template <typename T, int TT, int MAXT>
tdm_status dispatch(const CUtensorMap& map, const SolveArgs& args, const Cfg& cfg, cudaStream_t s) {
  if (cfg.tma) {
    switch (cfg.R) {
      case 8: return launch_t<T, 8, TT, MAXT, true>(map, args, cfg, s);
      case 16: return launch_t<T, 16, TT, MAXT, true>(map, args, cfg, s);
      case 32: return launch_t<T, 32, TT, MAXT, true>(map, args, cfg, s);
    }
  } else {
    switch (cfg.R) {
      case 8: return launch_t<T, 8, TT, MAXT, false>(map, args, cfg, s);
      case 16: return launch_t<T, 16, TT, MAXT, false>(map, args, cfg, s);
      case 32: return launch_t<T, 32, TT, MAXT, false>(map, args, cfg, s);
    }
  }
  return TDM_ERR_NOT_IMPLEMENTED;
}

// shared memory of a configuration; the binary32 solve keeps its A4 arrays in
// the pair layout, sized for 512 / R blocks
size_t cfg_smem(const Cfg& cfg, int t, bool fp64, bool tma) {
  const int tsize = fp64 ? 8 : 4;
  return fp64 ? smem_bytes(cfg.m, t, cfg.R, tsize, tma)
              : 128 + fbuf_bytes(cfg.m, t, cfg.R, tsize, tma) + coef_bytes(cfg.m, t, tsize) +
                    iface_offsets(cfg.R, 512 / cfg.R, false).bytes;
}

}  // namespace

// The cooperative binary64 solve for a plan of M blocks of t rows: the grid
// (whole groups) when it holds at least 1.2 times the CTAs that clusters of
// the same width can, else 0; *scr_bytes receives its scratch.
int tdm_plain_coop_choice(int M, int t, size_t* scr_bytes) {
  Cfg cfg;
  if (!choose_cfg(M, t, true, cfg) || cfg.C < 2) return 0;
  cfg.tma = true;
  cfg.smem = cfg_smem(cfg, t, true, true);
  if (cfg.smem > 227 * 1024) return 0;
  int blocks = 0, slots = 0;
  switch (cfg.R * 100 + t) {
    case 8 * 100 + 16: blocks = coop_blocks<8, 16, true>(cfg); slots = cluster_slots<8, 16, true>(cfg); break;
    case 16 * 100 + 16: blocks = coop_blocks<16, 16, true>(cfg); slots = cluster_slots<16, 16, true>(cfg); break;
    case 8 * 100 + 32: blocks = coop_blocks<8, 32, true>(cfg); slots = cluster_slots<8, 32, true>(cfg); break;
    case 16 * 100 + 32: blocks = coop_blocks<16, 32, true>(cfg); slots = cluster_slots<16, 32, true>(cfg); break;
  }
  const int grid = blocks / cfg.C * cfg.C;
  if (grid < cfg.C || (double)grid < 1.2 * (double)slots) return 0;
  *scr_bytes = sizeof(double) * (size_t)grid * 4 * cfg.R;
  return grid;
}

tdm_status tdm_launch_plain(tdm_plan_s* p, const void* F, int64_t ldF, void* X, int64_t ldX,
                            int64_t N, bool fp64, cudaStream_t s) {
  Cfg cfg;
  if (!choose_cfg(p->M, p->t, fp64, cfg)) return TDM_ERR_NOT_IMPLEMENTED;
  const int tsize = fp64 ? 8 : 4;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  cfg.tma = tdm_encode_tma_2d(&map, F, fp64, (uint64_t)N, (uint64_t)p->n, (uint64_t)ldF * tsize,
                              (uint32_t)cfg.R, (uint32_t)cfg.box_rows);
  cfg.smem = cfg_smem(cfg, p->t, fp64, cfg.tma);
  if (cfg.smem > 227 * 1024) {   // fall back to direct loads when the staging buffer does not fit
    cfg.tma = false;
    cfg.smem = cfg_smem(cfg, p->t, fp64, false);
  }
  SolveArgs args;
  args.F = F; args.X = X; args.ldF = ldF; args.ldX = ldX; args.N = N;
  args.coef = fp64 ? (const void*)p->coef64 : (const void*)p->coef32;
  args.rR = p->rR; args.rL = p->rL; args.err = p->dev_err;
  args.n = (int)p->n; args.M = p->M; args.m = cfg.m; args.C = cfg.C;
  args.ntiles = (int)((N + cfg.R - 1) / cfg.R);
  args.box_rows = cfg.box_rows;
  args.scr = p->coop64_scr;
  args.ctr = p->coop64_ctr;
  if (fp64 && p->coop64_grid > 0) {   // the cooperative form (chosen at prepare)
    if (p->t == 16) return dispatch_coop<16>(map, args, cfg, p->coop64_grid, s);
    return dispatch_coop<32>(map, args, cfg, p->coop64_grid, s);
  }
  if (fp64) {
    if (p->t == 16) return dispatch<double, 16, 512>(map, args, cfg, s);
    return dispatch<double, 32, 512>(map, args, cfg, s);
  }
  if (p->t == 16) return dispatch<float, 16, 512>(map, args, cfg, s);
  return dispatch<float, 32, 512>(map, args, cfg, s);
}
