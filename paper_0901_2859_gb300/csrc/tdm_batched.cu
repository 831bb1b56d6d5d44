// tdm_batched.cu -- many constant matrices, each with its own block of
// right-hand sides (the per-mode series of the Fourier method, Section 4,
// eqs. series_fft, poisson_end), solved by the refined persistent kernel.
//
// The series are grouped by the tile shape their size needs (right-hand sides
// per tile, blocks per CTA, CTAs per cluster); every group becomes one
// persistent launch over a device-resident work list of (series, tile) items.
// Work lists are built on the host on first use of an argument set and kept
// until one of their plans is destroyed, so repeated calls with the same
// arguments -- and replays of a CUDA graph that captured such a call -- upload
// nothing.
//
// Other precisions are served by one launch per series.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <list>
#include <mutex>
#include <vector>

#include "tdm_refine.cuh"

namespace {

struct ShapeClass {
  RefShape sh;
  int t = 0;
  int offset = 0, count = 0;   // range of the work list
};

struct WorkList {
  std::vector<uint64_t> key;
  RefItem* d_items = nullptr;
  RefItem* h_items = nullptr;   // pinned staging, alive as long as the list
  int device = 0;
  std::vector<ShapeClass> classes;
  ~WorkList() {
    if (d_items) cudaFree(d_items);
    if (h_items) cudaFreeHost(h_items);
  }
};

std::mutex g_mu;
std::list<WorkList*> g_cache;   // most recently used first

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

tdm_status build(WorkList* w, tdm_plan_s* const* ps, int count, const void* const* F, const int64_t* ldF,
                 void* const* X, const int64_t* ldX, const int64_t* N, cudaStream_t s) {
  struct Entry {
    int k;
    RefShape sh;
    double cost;
  };
  std::vector<Entry> es;
  for (int k = 0; k < count; k++) {
    if (N[k] == 0) continue;
    if (ldF[k] > kRefMaxLd || ldX[k] > kRefMaxLd) return TDM_ERR_NOT_IMPLEMENTED;
    RefShape sh;
    if (!tdm_refined_shape(ps[k]->M, ps[k]->t, ps[k]->tile_rhs, sh)) return TDM_ERR_NOT_IMPLEMENTED;
    es.push_back({k, sh, (double)ps[k]->n * (double)N[k]});
  }
  auto same = [](const RefShape& a, const RefShape& b) {
    return a.R == b.R && a.NT == b.NT && a.m == b.m && a.C == b.C;
  };
  // group by shape (and block rows), biggest series first inside a group
  std::stable_sort(es.begin(), es.end(), [&](const Entry& x, const Entry& y) {
    const int tx = ps[x.k]->t, ty = ps[y.k]->t;
    if (tx != ty) return tx < ty;
    if (x.sh.C != y.sh.C) return x.sh.C > y.sh.C;
    if (x.sh.R != y.sh.R) return x.sh.R > y.sh.R;
    if (x.sh.m != y.sh.m) return x.sh.m > y.sh.m;
    return x.cost > y.cost;
  });
  std::vector<RefItem> items;
  for (size_t i = 0; i < es.size(); i++) {
    const Entry& e = es[i];
    const int t = ps[e.k]->t;
    if (w->classes.empty() || !same(w->classes.back().sh, e.sh) || w->classes.back().t != t) {
      ShapeClass c;
      c.sh = e.sh;
      c.t = t;
      c.offset = (int)items.size();
      w->classes.push_back(c);
    }
    RefItem base = tdm_refined_item(ps[e.k], static_cast<const float*>(F[e.k]), ldF[e.k],
                                    static_cast<double*>(X[e.k]), ldX[e.k], N[e.k], e.k);
    const int ntiles = (int)((N[e.k] + e.sh.R - 1) / e.sh.R);
    for (int tile = 0; tile < ntiles; tile++) {
      base.tile = tile;
      items.push_back(base);
    }
    w->classes.back().count = (int)items.size() - w->classes.back().offset;
  }
  if (items.empty()) return TDM_OK;
  const size_t bytes = sizeof(RefItem) * items.size();
  TDM_CUDA_TRY(cudaMalloc(&w->d_items, bytes));
  TDM_CUDA_TRY(cudaMallocHost(&w->h_items, bytes));
  memcpy(w->h_items, items.data(), bytes);
  TDM_CUDA_TRY(cudaMemcpyAsync(w->d_items, w->h_items, bytes, cudaMemcpyHostToDevice, s));
  return TDM_OK;
}

}  // namespace

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
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<uint64_t> key = make_key(ps, count, F, ldF, X, ldX, N);
  std::lock_guard<std::mutex> g(g_mu);
  WorkList* w = nullptr;
  for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
    if ((*it)->device == dev && (*it)->key == key) {
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
    tdm_status st = build(w, ps, count, F, ldF, X, ldX, N, s);
    if (st != TDM_OK) {
      delete w;
      return st;
    }
    g_cache.push_front(w);
  }
  for (const ShapeClass& c : w->classes) {
    tdm_status st = tdm_refined_launch(c.sh, c.t, w->d_items + c.offset, nullptr, c.count, ps[0]->dev_err, s);
    if (st != TDM_OK) return st;
  }
  return TDM_OK;
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
