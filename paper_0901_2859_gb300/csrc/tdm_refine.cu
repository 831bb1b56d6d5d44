// tdm_refine.cu -- binary32 dichotomy solves with iterative refinement: F in
// binary32, X in binary64, accuracy of a binary64 solve (or better).
//
// Per tile of R right-hand sides (a cluster owns all n rows, as in the plain
// solve), with the tile's F kept in shared memory and the iterate x held in
// registers as a binary32 pair (x = xh + xl, ~48 significant bits):
//
//   x  = solve32(F)                                   (steps A2-A5, binary32)
//   repeat k times:
//     r_i = F_i - (A x)_i                             (error-free, see below)
//     x  += solve32(r)
//   X_i = xh_i + xl_i rounded once to binary64.
//
// The residual is formed in row-sum form.  With sigma_i = b_i + a_{i-1} + a_i
// and the fluxes E_i = a_i (x_{i+1} - x_i),
//     (A x)_i = sigma_i x_i - E_{i-1} + E_i,
// so  r_i = F_i - sigma_i x_i + E_{i-1} - E_i.  For the weakly dominant,
// ill-conditioned series of Section 4 the fluxes are small next to A's
// entries times x, the differences x_{i+1} - x_i are formed exactly from the
// pair representation, and the large terms E_{i-1} - E_i cancel exactly in
// Knuth's TwoSum; the residual's absolute error stays near 2^-48 |E| instead of
// 2^-24 |A||x|.  No binary64 instruction is issued per unknown except the
// final rounding of xh + xl.  Iterative refinement itself is not part of the
// paper's method; its correction solves are the paper's method in binary32.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "tdm_df.cuh"
#include "tdm_kernel_common.cuh"
#include "tdm_tma.cuh"

namespace {
using namespace tdmk;

struct RefineArgs {
  SolveArgs s;        // F (binary32), X (binary64), coefficients (binary32)
  const float* res;   // [n][8] residual coefficients: sigma and a split in binary32 parts
  int steps;          // refinement steps after the first solve
};

__host__ __device__ inline size_t refine_smem_bytes(int m, int t, int R) {
  const int rows = m * t;
  return 128 + (size_t)rows * R * 4          // F tile
         + (size_t)rows * R * 4              // low words of the iterate
         + (size_t)rows * kNCOEF * 4         // solve coefficients
         + (size_t)(rows + 1) * 4 * 4        // residual coefficients (sigma_h, sigma_l, a_h, a_l)
         + (size_t)4 * m * R * 4             // block edge values of x (first/last row, hi/lo)
         + (size_t)2 * m * R * 4 + 4 * R * 4 // convergence maxima (per block, per CTA x2 parity)
         + smem_bytes(m, t, R, 4, false) - 128 - coef_bytes(m, t, 4);
}

// Estimated relative error left after a correction d_k: ratio_k^2 / ratio_{k-1}
// (linear convergence), with ratio_k = max over columns of max|d_k| / max|x|;
// after the first correction, ratio_1 itself.
constexpr float kRefineTol = 1e-12f;

// max over columns of (max|d| / max|x|) over the whole cluster; every thread of
// every CTA gets the same value (exact maxima read in the same order).
template <int R>
__device__ __forceinline__ float cluster_ratio(const float* slot, int C, int tid, float* bcast) {
  if (tid < 32) {
    float q = 0.f;
    if (tid < R) {
      float md = 0.f, mx = 0.f;
      for (int cc = 0; cc < C; cc++) {
        md = fmaxf(md, ld_cluster_f32(slot + tid, (unsigned)cc));
        mx = fmaxf(mx, ld_cluster_f32(slot + R + tid, (unsigned)cc));
      }
      q = mx > 0.f ? md / mx : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) q = fmaxf(q, __shfl_xor_sync(0xffffffffu, q, o));
    if (tid == 0) *bcast = q;
  }
  __syncthreads();
  return *bcast;
}

// A5 of a correction solve: back substitution, correction with the separator
// values, and x += d in pair arithmetic (high words in registers, low words in
// shared memory at stride R); tracks max|d| and max|x| for the convergence test.
template <int R, int TT, bool FULL>
__device__ __forceinline__ void backward_update(const float (&g)[TT], const float* cf, int nrows, float xL,
                                                float xR, float (&xh)[TT], float* xlt, float& maxd,
                                                float& maxx) {
  float y = 0.f;
#pragma unroll
  for (int i = TT - 1; i >= 0; i--) {
    if (FULL || i < nrows) {
      float cc, invd, phl, phr;
      ld4(cf + i * kNCOEF + 4, cc, invd, phl, phr);
      y = fmaf(-cc, y, g[i]) * invd;
      const float d = fmaf(phr, xR, fmaf(phl, xL, y));
      const f2pair xn = df_add_f(f2pair{xh[i], xlt[i * R]}, d);
      xh[i] = xn.h;
      xlt[i * R] = xn.l;
      maxd = fmaxf(maxd, fabsf(d));
      maxx = fmaxf(maxx, fabsf(xn.h));
    }
  }
}

template <int R, int TT, bool TMA>
__global__ void __launch_bounds__(512, 1) k_solve_refined(const __grid_constant__ CUtensorMap tmF, const RefineArgs ra) {
  const SolveArgs& a = ra.s;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int wait_ok;
  __shared__ float ratio_s;
  const int m = a.m;
  const int rows_cta = m * TT;
  unsigned char* base = smem_raw + smem_align_pad(smem_raw);
  float* fbuf = reinterpret_cast<float*>(base);                         // [rows_cta][R]  F tile
  float* sxl = fbuf + (size_t)rows_cta * R;                             // [rows_cta][R]  low words of x
  float* scf = sxl + (size_t)rows_cta * R;                              // [rows_cta][8]
  float* sres = scf + (size_t)rows_cta * kNCOEF;                        // [rows_cta + 1][4]
  float* eFh = sres + (size_t)(rows_cta + 1) * 4;                       // [m][R] first-row x, hi
  float* eFl = eFh + m * R;
  float* eLh = eFl + m * R;                                             // [m][R] last-row x, hi
  float* eLl = eLh + m * R;
  float* redD = eLl + m * R;                                            // [m][R] max |d| per block
  float* redX = redD + m * R;                                           // [m][R] max |x| per block
  float* cvg = redX + m * R;                                            // [2 parity][2][R] per CTA, read remotely
  const Smem s = carve(reinterpret_cast<unsigned char*>(cvg + 4 * R), m, R, 4);

  const unsigned c = cluster_rank();
  const int tid = threadIdx.x;
  const int r = tid % R;
  const int bl = tid / R;
  const int b = (int)c * m + bl;
  const bool blk_ok = (bl < m) && (b < a.M);
  const int64_t row0 = (int64_t)b * TT;
  const int nrows = blk_ok ? (int)((a.n - row0) < TT ? (a.n - row0) : TT) : 0;   // rows that exist
  const int64_t cta_row0 = (int64_t)c * rows_cta;
  const int n = a.n;
  const float* __restrict__ coef = static_cast<const float*>(a.coef);
  double* __restrict__ X = static_cast<double*>(a.X);
  // steps > 0: exactly that many corrections; otherwise adaptive with a cap of 4
  const bool adaptive = ra.steps <= 0;
  const int cap = adaptive ? 4 : ra.steps;

  setup_ratios(a, s, c);
  for (int k = tid; k < rows_cta * kNCOEF / 4; k += blockDim.x) {
    const int64_t row = cta_row0 + (k * 4) / kNCOEF;
    float x = 0.f, y = 0.f, z = 0.f, w = 0.f;
    if (row < n) ld4(coef + cta_row0 * kNCOEF + (int64_t)k * 4, x, y, z, w);
    float* d = scf + (size_t)k * 4;
    d[0] = x; d[1] = y; d[2] = z; d[3] = w;
  }
  for (int k = tid; k <= rows_cta; k += blockDim.x) {   // rows cta_row0-1 .. cta_row0+rows_cta-1
    const int64_t row = cta_row0 - 1 + k;
    float sh = 0.f, sl = 0.f, ah = 0.f, al = 0.f;
    if (row >= 0 && row < n) {
      const float* q = ra.res + row * kNRES;
      sh = q[kS0]; sl = q[kS1]; ah = q[kA0]; al = q[kA1];
    }
    float* d = sres + (size_t)k * 4;
    d[0] = sh; d[1] = sl; d[2] = ah; d[3] = al;
  }
  if (TMA && tid == 0) tdm_mbar_init(&mbar, 1);
  __syncthreads();

  const int cluster_id = blockIdx.x / a.C;
  const int nclusters = gridDim.x / a.C;
  const uint32_t tile_bytes = (uint32_t)rows_cta * R * 4;
  const int nbox = rows_cta / a.box_rows;
  auto issue = [&](int tile) {
    tdm_mbar_expect_tx(&mbar, tile_bytes);
    for (int k = 0; k < nbox; k++)
      tdm_tma_load_2d(fbuf + (size_t)k * a.box_rows * R, &tmF, tile * R, (int)(cta_row0 + (int64_t)k * a.box_rows),
                      &mbar);
  };
  if (TMA && tid == 0 && cluster_id < a.ntiles) issue(cluster_id);

  uint32_t phase = 0u;
  bool abort = false;
  int parity = 0;
  for (int tile = cluster_id; tile < a.ntiles; tile += nclusters) {
    const int64_t col = (int64_t)tile * R + r;
    const bool col_ok = col < a.N;
    if constexpr (TMA) {
      if (!abort && !tdm_mbar_wait_cta(&mbar, phase, a.err, &wait_ok)) abort = true;
      phase ^= 1u;
    } else {   // direct coalesced loads into the tile buffer
      const float* __restrict__ F = static_cast<const float*>(a.F);
      float* dst = fbuf + (size_t)bl * TT * R + r;
#pragma unroll 4
      for (int i = 0; i < TT; i++) {
        const int64_t row = row0 + i;
        if (bl < m) dst[i * R] = (blk_ok && col_ok && row < n) ? F[row * a.ldF + col] : 0.f;
      }
      __syncthreads();
    }
    const float* Ft = fbuf + (size_t)bl * TT * R + r;
    float* xlt = sxl + (size_t)bl * TT * R + r;   // this thread's low words, stride R

    float xh[TT], g[TT];
#pragma unroll
    for (int i = 0; i < TT; i++) { xh[i] = 0.f; if (bl < m) xlt[i * R] = 0.f; }

    float ratio_prev = 1.f;
    int cpar = 0;
    for (int step = 0;; step++) {
      if (step == 0) {
#pragma unroll
        for (int i = 0; i < TT; i++) g[i] = blk_ok ? Ft[i * R] : 0.f;   // zeros beyond n
      } else {
        // ---- residual r = F - A x of the current iterate ------------------------
        // (threads beyond the CTA's m blocks only take part in the barriers)
        if (bl < m) {
          eFh[bl * R + r] = xh[0]; eFl[bl * R + r] = xlt[0];
          eLh[bl * R + r] = xh[TT - 1]; eLl[bl * R + r] = xlt[(TT - 1) * R];
        }
        cluster_barrier();
        if (adaptive && step >= 2) {   // converged after the previous correction?
          // after the first correction there is no contraction estimate yet: stop only if
          // the correction itself is below the tolerance
          const float ratio = cluster_ratio<R>(cvg + (cpar ^ 1) * 2 * R, a.C, tid, &ratio_s);
          const bool stop = (step == 2) ? (ratio <= kRefineTol) : (ratio * ratio <= kRefineTol * ratio_prev);
          ratio_prev = ratio;
          if (stop) break;
        }
        if (bl >= m) {
#pragma unroll
          for (int i = 0; i < TT; i++) g[i] = 0.f;
        } else {
        f2pair xm{0.f, 0.f}, xp{0.f, 0.f};   // x at rows row0-1 and row0+TT
        if (bl > 0) {
          xm = f2pair{eLh[(bl - 1) * R + r], eLl[(bl - 1) * R + r]};
        } else if (c > 0) {
          xm = f2pair{ld_cluster_f32(eLh + (m - 1) * R + r, c - 1), ld_cluster_f32(eLl + (m - 1) * R + r, c - 1)};
        }
        if (bl < m - 1) {
          xp = f2pair{eFh[(bl + 1) * R + r], eFl[(bl + 1) * R + r]};
        } else if ((int)c < a.C - 1) {
          xp = f2pair{ld_cluster_f32(eFh + r, c + 1), ld_cluster_f32(eFl + r, c + 1)};
        }
        // flux into the first row: E_{row0-1} = a_{row0-1} (x_row0 - x_{row0-1})
        const float* rc = sres + (size_t)(bl * TT) * 4;   // row0-1 at index bl*TT
        f2pair xi{xh[0], xlt[0]};
        f2pair Ep = df_mul(f2pair{rc[2], rc[3]}, df_diff(xi, xm));
#pragma unroll
        for (int i = 0; i < TT; i++) {
          float sh, sl, ah, al;
          ld4(rc + (i + 1) * 4, sh, sl, ah, al);
          const f2pair xn = (i + 1 < TT) ? f2pair{xh[i + 1], xlt[(i + 1) * R]} : xp;
          const f2pair E = df_mul(f2pair{ah, al}, df_diff(xn, xi));
          const f2pair S = df_mul(f2pair{sh, sl}, xi);
          const float Fi = Ft[i * R];   // bl < m here; rows beyond n hold zeros
          const f2pair w = two_sum_f(Ep.h, -E.h);
          const f2pair u = two_sum_f(Fi, w.h);
          const f2pair v = two_sum_f(u.h, -S.h);
          const float small = ((Ep.l - E.l) - S.l) + (w.l + u.l + v.l);
          g[i] = v.h + small;
          Ep = E;
          xi = xn;
        }
        }
      }

      // ---- binary32 dichotomy solve of g (A2-A5) ---------------------------------
      const float* cfb = scf + (size_t)bl * TT * kNCOEF;
      float bR = 0.f, bL = 0.f;
      if (nrows == TT) forward_pass<float, TT, true>(g, cfb, nrows, bR, bL);
      else forward_pass<float, TT, false>(g, cfb, nrows, bR, bL);
      if (bl < m) {
        s.betaR[bl * R + r] = tdm_f2d(bR);
        s.betaL[bl * R + r] = tdm_f2d(bL);
      }
      __syncthreads();
      separator_partials<float, R>(a, s, c, parity);
      parity ^= 1;
      float xL = 0.f, xR = 0.f;
      if (blk_ok) {
        if (b >= 1) xL = separator_value<float, R>(s, bl, r);
        if (b + 1 <= a.M - 1) xR = separator_value<float, R>(s, bl + 1, r);
      }
      float maxd = 0.f, maxx = 0.f;
      if (nrows == TT) backward_update<R, TT, true>(g, cfb, nrows, xL, xR, xh, xlt, maxd, maxx);
      else backward_update<R, TT, false>(g, cfb, nrows, xL, xR, xh, xlt, maxd, maxx);
      if (adaptive && step >= 1) {   // per-CTA, per-column maxima of |d| and |x| for the test
        if (bl < m) { redD[bl * R + r] = maxd; redX[bl * R + r] = maxx; }
        __syncthreads();
        if (tid < R) {
          float md = 0.f, mx = 0.f;
          for (int j = 0; j < m; j++) { md = fmaxf(md, redD[j * R + tid]); mx = fmaxf(mx, redX[j * R + tid]); }
          cvg[cpar * 2 * R + tid] = md;
          cvg[cpar * 2 * R + R + tid] = mx;
        }
        cpar ^= 1;
      }
      if (step == cap) {
        if (adaptive) {   // cap reached: record whether the last correction met the test
          cluster_barrier();
          const float ratio = cluster_ratio<R>(cvg + (cpar ^ 1) * 2 * R, a.C, tid, &ratio_s);
          if (tid == 0 && !(ratio * ratio <= kRefineTol * ratio_prev)) atomicExch(a.err, kDevErrNotConverged);
        }
        break;
      }
    }
    // this tile's F is no longer read: start loading the next tile
    if constexpr (TMA) {
      __syncthreads();
      if (tid == 0 && !abort && tile + nclusters < a.ntiles) {
        tdm_fence_proxy_async();
        issue(tile + nclusters);
      }
    }
    // ---- X = xh + xl rounded once to binary64 -------------------------------------
    if (col_ok) {
      double* p = X + row0 * a.ldX + col;
#pragma unroll
      for (int i = 0; i < TT; i++) {
        if (i < nrows) *p = tdm_f2d(xh[i]) + tdm_f2d(xlt[i * R]);
        p += a.ldX;
      }
    }
  }
  cluster_barrier();
}

struct RCfg {
  int R = 16, m = 0, C = 0, threads = 0, box_rows = 0;
  size_t smem = 0;
};

bool choose_rcfg(int M, int t, RCfg& cfg) {
  for (int R : {16, 8}) {
    const int m_max = 512 / R;
    const int C = (M + m_max - 1) / m_max;
    if (C > 16) continue;
    const int m = (M + C - 1) / C;
    int threads = ((m * R + 31) / 32) * 32;
    if (threads < 96) threads = 96;
    int g = 1;
    for (int d = 1; d <= m; d++)
      if (m % d == 0 && d * t <= 256) g = d;
    cfg.R = R; cfg.m = m; cfg.C = C; cfg.threads = threads; cfg.box_rows = g * t;
    cfg.smem = refine_smem_bytes(m, t, R);
    if (cfg.smem > 227 * 1024) continue;
    return true;
  }
  return false;
}

template <int R, int TT, bool TMA>
tdm_status launch_refined(const CUtensorMap& map, const RefineArgs& args, const RCfg& cfg, cudaStream_t s) {
  auto kern = k_solve_refined<R, TT, TMA>;
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t, int>, int> occ;
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
  const int nclusters = args.s.ntiles < maxc ? args.s.ntiles : maxc;
  lc.gridDim = dim3(nclusters * cfg.C);
  TDM_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, map, args));
  return TDM_OK;
}

}  // namespace

tdm_status tdm_launch_refined(tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX,
                              int64_t N, cudaStream_t s) {
  RCfg cfg;
  if (!choose_rcfg(p->M, p->t, cfg)) return TDM_ERR_NOT_IMPLEMENTED;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const bool tma = getenv("TDM_NO_TMA") == nullptr &&
                   tdm_encode_tma_2d(&map, F, false, (uint64_t)N, (uint64_t)p->n, (uint64_t)ldF * 4,
                                     (uint32_t)cfg.R, (uint32_t)cfg.box_rows);
  RefineArgs args;
  SolveArgs& a = args.s;
  a.F = F; a.X = X; a.ldF = ldF; a.ldX = ldX; a.N = N;
  a.coef = p->coef32;
  a.rR = p->rR; a.rL = p->rL; a.err = p->dev_err;
  a.n = (int)p->n; a.M = p->M; a.m = cfg.m; a.C = cfg.C;
  a.ntiles = (int)((N + cfg.R - 1) / cfg.R);
  a.box_rows = cfg.box_rows;
  args.res = p->res32;
  args.steps = p->refine_steps;
  switch (cfg.R * 100 + p->t) {
    case 1632: return tma ? launch_refined<16, 32, true>(map, args, cfg, s) : launch_refined<16, 32, false>(map, args, cfg, s);
    case 1616: return tma ? launch_refined<16, 16, true>(map, args, cfg, s) : launch_refined<16, 16, false>(map, args, cfg, s);
    case 832: return tma ? launch_refined<8, 32, true>(map, args, cfg, s) : launch_refined<8, 32, false>(map, args, cfg, s);
    case 816: return tma ? launch_refined<8, 16, true>(map, args, cfg, s) : launch_refined<8, 16, false>(map, args, cfg, s);
  }
  return TDM_ERR_NOT_IMPLEMENTED;
}
