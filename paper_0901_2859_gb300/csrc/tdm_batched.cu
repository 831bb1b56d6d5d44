// tdm_batched.cu -- many constant matrices, each with its own block of
// right-hand sides (the per-mode series of the Fourier method, Section 4,
// eqs. series_fft, poisson_end), solved by the refined persistent kernel.
//
// Four ways to lay the work out (tdm_set_batched_strategy; by default a rule
// picks the first for batches that need many launch classes, the second for
// those that need few, such as the equal-size modes of one Poisson problem):
//
//  * one launch per series: every series is solved by its own
//    single-series launch (the item's fields in kernel parameters, the leanest
//    form of the kernel), biggest series first, round robin over the caller's
//    stream and helper streams that fork from it and join it again, so that
//    small series that fill a few clusters run side by side;
//
//  * by cluster width: the series are grouped by the kernel shape their size
//    needs and by the CTAs per cluster of that shape; every group is one
//    persistent launch over a work list of (series, tile) items whose clusters
//    each take one tile at a time; the launches are spread over the streams
//    in the same way;
//
//  * grouped units: one launch per kernel shape.  Every series gets a group
//    of g CTAs (its single-series partition, rounded up to a power of two)
//    and is cut into tiles of R right-hand sides.  The clusters have as many
//    CTAs as the largest group; a cluster walks its own list of units, and in
//    a unit every aligned range of g ranks can solve a tile of a different
//    series.  The units are laid out on the host: the tiles of each series in
//    runs of consecutive units on the same ranks (one set-up of its
//    coefficients per run), each run placed where the ranks become free
//    first, biggest groups first.  All CTAs of a cluster pass the same cluster
//    barriers in every unit, so a unit's tiles share one schedule of
//    corrections: series with different schedules (fixed counts, the
//    speculative test) go to different launches.
//
//  * cooperative runs: one cooperative launch per kernel shape over every CTA
//    the GPU holds, with groups of consecutive CTAs in place of clusters
//    (see build_coop), so that no CTA slot is lost to cluster placement.
//
// All of them give every series the result of its own tdm_solve, bit for bit
// (the grouped units differ only where a tile is solved again, see
// tdm_set_batched_strategy).  Work lists are built on the host on first use of
// an argument set and kept until one of their plans is destroyed, so repeated
// calls with the same arguments -- and replays of a CUDA graph that captured
// such a call -- upload nothing.
//
// Other precisions are served by one launch per series.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <list>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tdm_refine.cuh"

namespace {

struct GroupedLaunch {
  RefShape sh;        // the kernel's shape; C = CTAs per cluster
  int t = 0;
  int nclusters = 0;  // grouped: clusters; list: items; cooperative: CTAs
  bool grouped = false;
  bool coop = false;  // a cooperative launch over runs
  int nruns = 0;
  size_t items_off = 0, units_off = 0, ustart_off = 0;   // byte offsets into the work list buffer
  size_t runs_off = 0, scr_off = 0, ctr_off = 0;         // cooperative: runs, scratch, counters
};

// 0: by cluster width, 1: grouped units, 2: one launch per series, 3: by rule, 4: cooperative runs
std::atomic<int> g_strategy{3};

struct WorkList {
  std::vector<uint64_t> key;
  int strategy = 0;
  unsigned char* d_buf = nullptr;
  unsigned char* h_buf = nullptr;   // pinned staging, alive as long as the list
  int device = 0;
  std::vector<GroupedLaunch> launches;
  ~WorkList() {
    if (d_buf) cudaFree(d_buf);
    if (h_buf) cudaFreeHost(h_buf);
  }
};

std::mutex g_mu;
std::list<WorkList*> g_cache;   // most recently used first

// the rule's limit: batches needing at most this many (shape, cluster width)
// launches run by cluster width, larger mixes one launch per series
constexpr size_t kRuleClasses = 4;

std::vector<uint64_t> make_key(tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                               void* const* X, const int64_t* ldX, const int64_t* N) {
  std::vector<uint64_t> k;
  k.reserve((size_t)count * 7);
  for (int i = 0; i < count; i++) {
    k.push_back((uint64_t)(uintptr_t)ps[i]);
    k.push_back((uint64_t)(uintptr_t)F[i]);
    k.push_back((uint64_t)ldF[i]);
    k.push_back((uint64_t)(uintptr_t)X[i]);
    k.push_back((uint64_t)ldX[i]);
    k.push_back((uint64_t)N[i]);
    k.push_back((uint64_t)ps[i]->refine_steps);
  }
  return k;
}

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// the schedule of corrections a series' tiles follow: k >= 1 fixed
// corrections, 0 the speculative test, -1 the fixed retry count
int schedule_of(const tdm_plan_s* p) {
  if (p->refine_steps >= 1) return p->refine_steps;
  return p->contraction < 1.f ? 0 : -1;
}

struct Series {
  int k;             // argument index
  int g, m;          // group CTAs, blocks per CTA
  int tiles;         // ceil(N / R)
  int first_item;    // index of its tile 0 in the launch's items
};

// Lays out the units of one launch: cursor[cl * C + q] is the number of units
// rank q of cluster cl is busy for.  Returns the unit table [units][kUnitW]
// (item indices, `null_item` where a rank has nothing) and the first unit of
// every cluster.
void lay_out(std::vector<Series>& ser, int C, int ncl, int null_item, std::vector<int>& units,
             std::vector<int>& ustart) {
  int64_t work = 0;
  for (const Series& s : ser) work += (int64_t)s.tiles * s.g;
  const int64_t target = (work + (int64_t)ncl * C - 1) / ((int64_t)ncl * C);   // units per rank if perfectly even
  const int run_cap = (int)std::max<int64_t>(1, (target + 7) / 8);
  std::vector<int64_t> cursor((size_t)ncl * C, 0);
  struct Run {
    int cl, q, g, start, len, item0;
  };
  std::vector<Run> runs;
  std::stable_sort(ser.begin(), ser.end(), [](const Series& a, const Series& b) {
    if (a.g != b.g) return a.g > b.g;
    return a.tiles > b.tiles;
  });
  for (const Series& s : ser) {
    int done = 0;
    while (done < s.tiles) {
      int best_cl = 0, best_q = 0;
      int64_t best = INT64_MAX;
      for (int cl = 0; cl < ncl; cl++)
        for (int q = 0; q < C; q += s.g) {
          int64_t st = 0;
          for (int j = 0; j < s.g; j++) st = std::max(st, cursor[(size_t)cl * C + q + j]);
          if (st < best) {
            best = st;
            best_cl = cl;
            best_q = q;
          }
        }
      int64_t len = std::min<int64_t>(s.tiles - done, run_cap);
      if (best < target) len = std::min<int64_t>(len, std::max<int64_t>(1, target - best));
      runs.push_back({best_cl, best_q, s.g, (int)best, (int)len, s.first_item + done});
      for (int j = 0; j < s.g; j++) cursor[(size_t)best_cl * C + best_q + j] = best + len;
      done += (int)len;
    }
  }
  ustart.assign(ncl + 1, 0);
  for (int cl = 0; cl < ncl; cl++) {
    int64_t u = 0;
    for (int q = 0; q < C; q++) u = std::max(u, cursor[(size_t)cl * C + q]);
    ustart[cl + 1] = ustart[cl] + (int)u;
  }
  units.assign((size_t)ustart[ncl] * kUnitW, null_item);
  for (const Run& r : runs)
    for (int i = 0; i < r.len; i++)
      for (int j = 0; j < r.g; j++)
        units[((size_t)ustart[r.cl] + r.start + i) * kUnitW + r.q + j] = r.item0 + i;
}

tdm_status build(WorkList* w, tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                 void* const* X, const int64_t* ldX, const int64_t* N, cudaStream_t s) {
  const bool grouped = w->strategy == 1;
  // launches by (block rows, tile width, threads, table placement, schedule
  // for grouped units / CTAs per cluster for lists)
  std::map<std::tuple<int, int, int, int, int>, std::vector<int>> by_launch;
  for (int k = 0; k < count; k++) {
    if (N[k] == 0) continue;
    if (ldF[k] > kRefMaxLd || ldX[k] > kRefMaxLd) return TDM_ERR_NOT_IMPLEMENTED;
    RefShape sh;
    if (!tdm_refined_shape(ps[k]->M, ps[k]->t, ps[k]->tile_rhs, sh)) return TDM_ERR_NOT_IMPLEMENTED;
    by_launch[std::make_tuple(ps[k]->t, sh.R, sh.NT, sh.sm_coef ? 1 : 0, grouped ? schedule_of(ps[k]) : -sh.C)]
        .push_back(k);
  }
  std::vector<RefItem> items;
  std::vector<int> all_units, all_ustart;
  struct Pending {
    GroupedLaunch gl;
    size_t items0, units0, ustart0;
  };
  std::vector<Pending> pend;
  for (auto& kv : by_launch) {
    const int t = std::get<0>(kv.first), R = std::get<1>(kv.first), NT = std::get<2>(kv.first);
    const bool smc = std::get<3>(kv.first) != 0;
    if (!grouped) {   // one list launch: the series' items, biggest series first
      std::vector<int> ks = kv.second;
      std::stable_sort(ks.begin(), ks.end(), [&](int x, int y) {
        return (double)ps[x]->n * (double)N[x] > (double)ps[y]->n * (double)N[y];
      });
      GroupedLaunch gl;
      gl.t = t;
      const size_t items0 = items.size();
      for (int k : ks) {
        RefShape sh;
        tdm_refined_shape(ps[k]->M, ps[k]->t, ps[k]->tile_rhs, sh);
        gl.sh = sh;
        RefItem it = tdm_refined_item(ps[k], static_cast<const float*>(F[k]), ldF[k], static_cast<double*>(X[k]),
                                      ldX[k], N[k], k, sh);
        const int tiles = (int)((N[k] + R - 1) / R);
        for (int tile = 0; tile < tiles; tile++) {
          it.tile = tile;
          items.push_back(it);
        }
      }
      gl.sh.m = NT / R;
      gl.sh.threads = ((gl.sh.m * R + 31) / 32) * 32;
      gl.nclusters = (int)(items.size() - items0);
      pend.push_back({gl, items0, all_units.size(), all_ustart.size()});
      continue;
    }
    std::vector<Series> ser;
    int C = 1;
    const size_t items0 = items.size();
    for (int k : kv.second) {
      RefShape sh;
      tdm_refined_shape(ps[k]->M, ps[k]->t, ps[k]->tile_rhs, sh);
      Series e;
      e.k = k;
      // the single-series partition (sh.C CTAs of sh.m blocks), in a group
      // rounded up to a power of two whose extra CTAs own no block: the same
      // arithmetic as a solve of the series alone, bit for bit
      e.g = pow2_at_least(sh.C);
      e.m = sh.m;
      e.tiles = (int)((N[k] + R - 1) / R);
      e.first_item = (int)(items.size() - items0);
      C = std::max(C, e.g);
      sh.m = e.m;
      sh.C = e.g;
      RefItem it = tdm_refined_item(ps[k], static_cast<const float*>(F[k]), ldF[k], static_cast<double*>(X[k]),
                                    ldX[k], N[k], k, sh);
      for (int tile = 0; tile < e.tiles; tile++) {
        it.tile = tile;
        items.push_back(it);
      }
      ser.push_back(e);
    }
    // the null item: no rows, no columns, the launch's schedule
    RefItem nul = items[items0];
    nul.N = 0;
    nul.n = 0;
    nul.M = 0;
    nul.m = 1;
    nul.g = 1;
    nul.tile = 0;
    nul.series = -2;
    const int null_item = (int)(items.size() - items0);
    items.push_back(nul);
    GroupedLaunch gl;
    gl.t = t;
    gl.grouped = true;
    gl.sh.R = R;
    gl.sh.NT = NT;
    gl.sh.C = C;
    gl.sh.m = NT / R;
    gl.sh.threads = NT;
    gl.sh.sm_coef = smc;
    gl.sh.smem = 0;
    {   // the shared memory the shape's kernel needs (the rule's shape of the first series)
      RefShape sh;
      tdm_refined_shape(ps[kv.second[0]]->M, t, ps[kv.second[0]]->tile_rhs, sh);
      gl.sh.smem = sh.smem;
    }
    const int maxc = tdm_refined_max_clusters(gl.sh, t);
    if (maxc < 1) return TDM_ERR_NOT_IMPLEMENTED;
    int64_t work = 0;
    for (const Series& e : ser) work += (int64_t)e.tiles * e.g;
    gl.nclusters = (int)std::min<int64_t>(maxc, std::max<int64_t>(1, (work + C - 1) / C));
    std::vector<int> units, ustart;
    lay_out(ser, C, gl.nclusters, null_item, units, ustart);
    pend.push_back({gl, items0, all_units.size(), all_ustart.size()});
    all_units.insert(all_units.end(), units.begin(), units.end());
    all_ustart.insert(all_ustart.end(), ustart.begin(), ustart.end());
  }
  if (items.empty()) return TDM_OK;
  const size_t items_bytes = sizeof(RefItem) * items.size();
  const size_t units_bytes = sizeof(int) * all_units.size();
  const size_t ustart_bytes = sizeof(int) * all_ustart.size();
  const size_t off_units = (items_bytes + 255) / 256 * 256;
  const size_t off_ustart = off_units + (units_bytes + 255) / 256 * 256;
  const size_t bytes = off_ustart + ustart_bytes;
  TDM_CUDA_TRY(cudaMalloc(&w->d_buf, bytes));
  TDM_CUDA_TRY(cudaMallocHost(&w->h_buf, bytes));
  memcpy(w->h_buf, items.data(), items_bytes);
  if (units_bytes) memcpy(w->h_buf + off_units, all_units.data(), units_bytes);
  memcpy(w->h_buf + off_ustart, all_ustart.data(), ustart_bytes);
  for (Pending& pd : pend) {
    pd.gl.items_off = sizeof(RefItem) * pd.items0;
    pd.gl.units_off = off_units + sizeof(int) * pd.units0;
    pd.gl.ustart_off = off_ustart + sizeof(int) * pd.ustart0;
    w->launches.push_back(pd.gl);
  }
  TDM_CUDA_TRY(cudaMemcpyAsync(w->d_buf, w->h_buf, bytes, cudaMemcpyHostToDevice, s));
  return TDM_OK;
}

// Helper streams of a device for the list launches (created on first use,
// kept for the life of the process), and the events that fork them from the
// caller's stream and join them back.
struct Helpers {
  static constexpr int kStreams = 3;
  cudaStream_t st[kStreams] = {};
  cudaEvent_t fork = nullptr, join[kStreams] = {};
  bool ok = false;
};
Helpers* helpers_of(int dev) {
  static Helpers h[64];
  if (dev < 0 || dev >= 64) return nullptr;
  Helpers& x = h[dev];
  if (!x.ok) {
    bool good = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; good && i < Helpers::kStreams; i++)
      good = cudaStreamCreateWithFlags(&x.st[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&x.join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!good) {
      (void)cudaGetLastError();
      return nullptr;
    }
    x.ok = true;
  }
  return &x;
}

// Cooperative runs: one launch per kernel shape over all CTAs the device
// holds.  Every series keeps its single-series partition (g = its CTAs per
// cluster, m its blocks per CTA) and is cut into runs of consecutive tiles;
// a run goes to the window of g consecutive CTAs that becomes free first
// (biggest groups first), so the runs that share a CTA are ordered by their
// start on every CTA alike and no group waits on a group that waits on it.
tdm_status build_coop(WorkList* w, tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                      void* const* X, const int64_t* ldX, const int64_t* N, cudaStream_t s) {
  std::map<std::tuple<int, int, int, int>, std::vector<int>> by_shape;
  for (int k = 0; k < count; k++) {
    if (N[k] == 0) continue;
    if (ldF[k] > kRefMaxLd || ldX[k] > kRefMaxLd) return TDM_ERR_NOT_IMPLEMENTED;
    RefShape sh;
    if (!tdm_refined_shape(ps[k]->M, ps[k]->t, ps[k]->tile_rhs, sh)) return TDM_ERR_NOT_IMPLEMENTED;
    by_shape[std::make_tuple(ps[k]->t, sh.R, sh.NT, sh.sm_coef ? 1 : 0)].push_back(k);
  }
  std::vector<RefItem> items;
  std::vector<RefRun> runs;
  std::vector<int> rlist, rstart;
  struct Pending {
    GroupedLaunch gl;
    size_t items0, runs0, rlist0, rstart0, scr_floats, ctr0;
  };
  std::vector<Pending> pend;
  size_t scr_total = 0, ctr_total = 0;
  for (auto& kv : by_shape) {
    const int t = std::get<0>(kv.first), R = std::get<1>(kv.first);
    RefShape lsh;
    tdm_refined_shape(ps[kv.second[0]]->M, t, ps[kv.second[0]]->tile_rhs, lsh);
    lsh.threads = lsh.NT;
    const int P = tdm_refined_coop_runs_grid(lsh, t);
    if (P < 16) return TDM_ERR_NOT_IMPLEMENTED;
    struct S {
      int k, g, tiles, item0;
    };
    std::vector<S> ser;
    const size_t items0 = items.size();
    int64_t work = 0;
    for (int k : kv.second) {
      RefShape sh;
      tdm_refined_shape(ps[k]->M, t, ps[k]->tile_rhs, sh);
      RefItem it = tdm_refined_item(ps[k], static_cast<const float*>(F[k]), ldF[k], static_cast<double*>(X[k]),
                                    ldX[k], N[k], k, sh);
      const int tiles = (int)((N[k] + R - 1) / R);
      ser.push_back({k, sh.C, tiles, (int)(items.size() - items0)});
      for (int tile = 0; tile < tiles; tile++) {
        it.tile = tile;
        items.push_back(it);
      }
      work += (int64_t)tiles * sh.C;
    }
    std::stable_sort(ser.begin(), ser.end(), [](const S& a, const S& b) {
      if (a.g != b.g) return a.g > b.g;
      return a.tiles > b.tiles;
    });
    const int64_t target = (work + P - 1) / P;
    const int run_cap = (int)std::max<int64_t>(1, (target + 7) / 8);
    std::vector<int64_t> cursor(P, 0);
    struct Placed {
      int64_t start;
      int run;
    };
    std::vector<std::vector<Placed>> per_cta(P);
    const size_t runs0 = runs.size();
    for (const S& e : ser) {
      int done = 0;
      while (done < e.tiles) {
        int best_p = 0;
        int64_t best = INT64_MAX;
        for (int p0 = 0; p0 + e.g <= P; p0++) {
          int64_t st = 0;
          for (int j = 0; j < e.g; j++) st = std::max(st, cursor[p0 + j]);
          if (st < best) {
            best = st;
            best_p = p0;
          }
        }
        int64_t len = std::min<int64_t>(e.tiles - done, run_cap);
        if (best < target) len = std::min<int64_t>(len, std::max<int64_t>(1, target - best));
        const int rid = (int)(runs.size() - runs0);
        runs.push_back({e.item0 + done, (int)len, best_p, e.g});
        for (int j = 0; j < e.g; j++) {
          cursor[best_p + j] = best + len;
          per_cta[best_p + j].push_back({best, rid});
        }
        done += (int)len;
      }
    }
    const size_t rlist0 = rlist.size(), rstart0 = rstart.size();
    for (int q = 0; q < P; q++) {
      std::stable_sort(per_cta[q].begin(), per_cta[q].end(),
                       [](const Placed& a, const Placed& b) { return a.start < b.start; });
      rstart.push_back((int)(rlist.size() - rlist0));
      for (const Placed& pl : per_cta[q]) rlist.push_back(pl.run);
    }
    rstart.push_back((int)(rlist.size() - rlist0));
    GroupedLaunch gl;
    gl.sh = lsh;
    gl.t = t;
    gl.coop = true;
    gl.nclusters = P;
    gl.nruns = (int)(runs.size() - runs0);
    const size_t scr_floats = tdm_refined_coop_scratch(lsh, P) / sizeof(float);
    pend.push_back({gl, items0, runs0, rlist0, rstart0, scr_floats, ctr_total});
    scr_total += scr_floats;
    ctr_total += (size_t)32 * gl.nruns;
  }
  if (items.empty()) return TDM_OK;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_items = sizeof(RefItem) * items.size(), b_runs = sizeof(RefRun) * runs.size();
  const size_t b_rlist = sizeof(int) * rlist.size(), b_rstart = sizeof(int) * rstart.size();
  const size_t o_runs = up(b_items), o_rlist = o_runs + up(b_runs), o_rstart = o_rlist + up(b_rlist);
  const size_t o_scr = o_rstart + up(b_rstart), o_ctr = o_scr + up(sizeof(float) * scr_total);
  const size_t upload = o_scr, bytes = o_ctr + sizeof(unsigned) * ctr_total;
  TDM_CUDA_TRY(cudaMalloc(&w->d_buf, bytes));
  TDM_CUDA_TRY(cudaMallocHost(&w->h_buf, upload));
  memcpy(w->h_buf, items.data(), b_items);
  memcpy(w->h_buf + o_runs, runs.data(), b_runs);
  memcpy(w->h_buf + o_rlist, rlist.data(), b_rlist);
  memcpy(w->h_buf + o_rstart, rstart.data(), b_rstart);
  size_t scr_at = o_scr;
  for (Pending& pd : pend) {
    pd.gl.items_off = sizeof(RefItem) * pd.items0;
    pd.gl.runs_off = o_runs + sizeof(RefRun) * pd.runs0;
    pd.gl.units_off = o_rlist + sizeof(int) * pd.rlist0;
    pd.gl.ustart_off = o_rstart + sizeof(int) * pd.rstart0;
    pd.gl.scr_off = scr_at;
    scr_at += sizeof(float) * pd.scr_floats;
    pd.gl.ctr_off = o_ctr + sizeof(unsigned) * pd.ctr0;
    w->launches.push_back(pd.gl);
  }
  TDM_CUDA_TRY(cudaMemcpyAsync(w->d_buf, w->h_buf, upload, cudaMemcpyHostToDevice, s));
  return TDM_OK;
}

}  // namespace

tdm_status tdm_set_batched_strategy(int strategy) {
  if (strategy < 0 || strategy > 4) return TDM_ERR_INVALID_ARG;
  g_strategy.store(strategy);
  return TDM_OK;
}

static tdm_status launch_batched_refined(tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                                        void* const* X, const int64_t* ldX, const int64_t* N, cudaStream_t s);

tdm_status tdm_launch_batched(tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                              void* const* X, const int64_t* ldX, const int64_t* N, tdm_precision prec,
                              cudaStream_t s) {
  if (prec != TDM_FP32_REFINED) {   // one launch per series
    for (int k = 0; k < count; k++) {
      if (N[k] == 0) continue;
      tdm_status st = tdm_launch_solve(ps[k], F[k], ldF[k], X[k], ldX[k], N[k], prec, s);
      if (st != TDM_OK) return st;
    }
    return TDM_OK;
  }
  // Series beyond one cluster (two-level plans) are solved one after the
  // other by their own two-level solve; the others share the batched layout.
  std::vector<tdm_plan_s*> ps1;
  std::vector<const void*> F1;
  std::vector<void*> X1;
  std::vector<int64_t> ldF1, ldX1, N1;
  for (int k = 0; k < count; k++) {
    if (N[k] > 0 && ps[k]->nseg > 0) continue;
    ps1.push_back(ps[k]);
    F1.push_back(F[k]);
    X1.push_back(X[k]);
    ldF1.push_back(ldF[k]);
    ldX1.push_back(ldX[k]);
    N1.push_back(N[k]);
  }
  if ((int)ps1.size() < count) {
    tdm_status st = ps1.empty() ? TDM_OK
                                : launch_batched_refined(ps1.data(), (int)ps1.size(), F1.data(), ldF1.data(),
                                                         X1.data(), ldX1.data(), N1.data(), s);
    for (int k = 0; k < count && st == TDM_OK; k++)
      if (N[k] > 0 && ps[k]->nseg > 0) st = tdm_launch_solve(ps[k], F[k], ldF[k], X[k], ldX[k], N[k], prec, s);
    return st;
  }
  return launch_batched_refined(ps, count, F, ldF, X, ldX, N, s);
}

static tdm_status launch_batched_refined(tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                                        void* const* X, const int64_t* ldX, const int64_t* N, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  int strategy = g_strategy.load();
  if (strategy == 3) {   // by rule: few launch classes -> by cluster width, else one launch per series
    std::vector<std::tuple<int, int, int, int>> cls;
    for (int k = 0; k < count; k++) {
      RefShape sh;
      if (N[k] == 0 || !tdm_refined_shape(ps[k]->M, ps[k]->t, ps[k]->tile_rhs, sh)) continue;
      const auto c = std::make_tuple(ps[k]->t, sh.R, sh.NT, sh.C);
      if (std::find(cls.begin(), cls.end(), c) == cls.end()) cls.push_back(c);
    }
    strategy = cls.size() <= kRuleClasses ? 0 : 2;
  }
  if (strategy == 2) {   // one single-series launch per series, round robin over the streams
    std::lock_guard<std::mutex> g(g_mu);
    Helpers* hp = helpers_of(dev);
    const int nstreams = hp ? 1 + Helpers::kStreams : 1;
    if (hp) {
      TDM_CUDA_TRY(cudaEventRecord(hp->fork, s));
      for (int i = 0; i < Helpers::kStreams; i++) TDM_CUDA_TRY(cudaStreamWaitEvent(hp->st[i], hp->fork, 0));
    }
    std::vector<int> ks;
    for (int k = 0; k < count; k++)
      if (N[k] > 0) ks.push_back(k);
    std::stable_sort(ks.begin(), ks.end(), [&](int x, int y) {
      return (double)ps[x]->n * (double)N[x] > (double)ps[y]->n * (double)N[y];
    });
    tdm_status st = TDM_OK;
    for (size_t i = 0; i < ks.size() && st == TDM_OK; i++) {
      const int k = ks[i];
      cudaStream_t ls = (i % nstreams) == 0 ? s : hp->st[(i % nstreams) - 1];
      st = tdm_launch_refined(ps[k], static_cast<const float*>(F[k]), ldF[k], static_cast<double*>(X[k]), ldX[k],
                              N[k], ls, false);
    }
    if (hp) {
      for (int i = 0; i < Helpers::kStreams; i++) {
        TDM_CUDA_TRY(cudaEventRecord(hp->join[i], hp->st[i]));
        TDM_CUDA_TRY(cudaStreamWaitEvent(s, hp->join[i], 0));
      }
    }
    return st;
  }
  std::vector<uint64_t> key = make_key(ps, count, F, ldF, X, ldX, N);
  std::lock_guard<std::mutex> g(g_mu);
  WorkList* w = nullptr;
  for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
    if ((*it)->device == dev && (*it)->strategy == strategy && (*it)->key == key) {
      w = *it;
      g_cache.erase(it);
      g_cache.push_front(w);
      break;
    }
  }
  if (!w) {
    w = new WorkList();
    w->key = key;
    w->device = dev;
    w->strategy = strategy;
    tdm_status st = strategy == 4 ? build_coop(w, ps, count, F, ldF, X, ldX, N, s)
                                  : build(w, ps, count, F, ldF, X, ldX, N, s);
    if (st != TDM_OK) {
      delete w;
      return st;
    }
    g_cache.push_front(w);
  }
  const int nl = (int)w->launches.size();
  Helpers* hp = nl > 1 && strategy != 4 ? helpers_of(dev) : nullptr;
  const int nstreams = hp ? 1 + Helpers::kStreams : 1;
  if (hp) {   // fork
    TDM_CUDA_TRY(cudaEventRecord(hp->fork, s));
    for (int i = 0; i < Helpers::kStreams; i++) TDM_CUDA_TRY(cudaStreamWaitEvent(hp->st[i], hp->fork, 0));
  }
  tdm_status st = TDM_OK;
  for (int i = 0; i < nl && st == TDM_OK; i++) {
    const GroupedLaunch& gl = w->launches[i];
    cudaStream_t ls = (i % nstreams) == 0 ? s : hp->st[(i % nstreams) - 1];
    const RefItem* items = reinterpret_cast<const RefItem*>(w->d_buf + gl.items_off);
    if (gl.coop)   // a cooperative grid takes the whole GPU: on the caller's stream, in order
      st = tdm_refined_launch_coop_runs(gl.sh, gl.t, items, reinterpret_cast<const RefRun*>(w->d_buf + gl.runs_off),
                                        reinterpret_cast<const int*>(w->d_buf + gl.units_off),
                                        reinterpret_cast<const int*>(w->d_buf + gl.ustart_off), gl.nruns, gl.nclusters,
                                        reinterpret_cast<float*>(w->d_buf + gl.scr_off),
                                        reinterpret_cast<unsigned*>(w->d_buf + gl.ctr_off), ps[0]->dev_err, s);
    else if (gl.grouped)
      st = tdm_refined_launch_grouped(gl.sh, gl.t, items, reinterpret_cast<const int*>(w->d_buf + gl.units_off),
                                      reinterpret_cast<const int*>(w->d_buf + gl.ustart_off), gl.nclusters,
                                      ps[0]->dev_err, ls);
    else
      st = tdm_refined_launch(gl.sh, gl.t, items, nullptr, gl.nclusters, ps[0]->dev_err, ls);
  }
  if (hp) {   // join (also after a failed launch: the helpers never stay forked)
    for (int i = 0; i < Helpers::kStreams; i++) {
      TDM_CUDA_TRY(cudaEventRecord(hp->join[i], hp->st[i]));
      TDM_CUDA_TRY(cudaStreamWaitEvent(s, hp->join[i], 0));
    }
  }
  return st;
}

// Drops the cached work lists that refer to plan p (called by tdm_destroy after
// the plan's work has finished).
void tdm_batched_forget(const tdm_plan_s* p) {
  std::lock_guard<std::mutex> g(g_mu);
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    bool uses = false;
    for (size_t i = 0; i < (*it)->key.size(); i += 7)
      if ((*it)->key[i] == (uint64_t)(uintptr_t)p) { uses = true; break; }
    if (uses) {
      delete *it;
      it = g_cache.erase(it);
    } else {
      ++it;
    }
  }
}
