// tdm_noalloc.cu -- tdm_solve_batched_noalloc: the batched refined solve with
// its work list in a fixed, statically sized device array instead of memory
// obtained from cudaMalloc.
//
// Who cannot allocate, and why:
//  - a caller whose device memory is held by its own pool (a framework's
//    caching allocator that has reserved most of HBM): a cudaMalloc inside the
//    solve can fail with out-of-memory although the pool has room;
//  - a caller in a time-stepping loop that overlaps copies and solves on
//    several streams: cudaMalloc, cudaMallocHost and the cudaFree that later
//    releases them may synchronize the device and stall the other streams;
//  - a caller that passes new F / X pointers on every call (buffers rotated
//    from its pool): the cached path of tdm_solve_batched builds and keeps one
//    work list per distinct argument set until a plan is destroyed, so its
//    memory grows with every new set.
//
// This path never allocates: the work list is staged in a static host array
// and copied into g_tiles, a static __device__ array of kMaxTiles items.  The
// refined kernel is the one the other solves use; only where its work items
// live differs.
//
// Sharing: every call on a device uses the same g_tiles, which keeps the last
// call's items.  No word of it needs to start at zero: each call writes every
// item its launches read, in stream order before those launches, so what an
// earlier call left there is never read.  Calls that overlap on the device
// (issued on different streams without ordering between them, or from several
// host threads on different streams) race on g_tiles and may solve each
// other's tiles; serialize them on one stream.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "tdm_refine.cuh"

tdm_status tdm_validate_solve(const tdm_plan_s* h, const void* F, int64_t ldF, const void* X, int64_t ldX,
                              int64_t N, tdm_precision prec);

namespace {

constexpr int kMaxTiles = TDM_NOALLOC_MAX_TILES;   // 4096 items x 96 B = 384 KiB per device
constexpr int kMaxDevices = 64;

static_assert(sizeof(RefItem) == 96, "work item layout");

static __device__ __align__(256) RefItem g_tiles[kMaxTiles];

struct Entry {
  int k;          // series number
  int t;          // block rows of its plan
  RefShape sh;    // tile shape of the refined kernel
  int tiles;      // ceil(N / R)
  double cost;    // n * N, biggest first inside a shape
};

std::mutex g_mu;                       // guards the host staging arrays and the set-up table
RefItem g_stage[kMaxTiles];            // host staging of one call's work list
Entry g_entries[kMaxTiles];            // non-empty series of one call (each has >= 1 tile)
RefItem* g_dev_ptr[kMaxDevices];       // address of g_tiles on each device, once set up
bool g_ready[kMaxDevices];

// Set-up, once per device, with that device current: the device address of
// g_tiles.  (The first use of the symbol also loads this module's device code
// on that device.)
tdm_status device_tiles(int dev, RefItem** out) {
  if (dev < 0 || dev >= kMaxDevices) return TDM_ERR_INVALID_ARG;
  if (!g_ready[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_tiles);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return TDM_ERR_CUDA;
    }
    g_dev_ptr[dev] = static_cast<RefItem*>(p);
    g_ready[dev] = true;
  }
  *out = g_dev_ptr[dev];
  return TDM_OK;
}

struct CurrentDevice {
  int prev = -1;
  explicit CurrentDevice(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~CurrentDevice() { if (prev >= 0) cudaSetDevice(prev); }
};

bool same_shape(const Entry& x, const Entry& y) {
  return x.t == y.t && x.sh.R == y.sh.R && x.sh.NT == y.sh.NT && x.sh.m == y.sh.m && x.sh.C == y.sh.C;
}

}  // namespace

extern "C" tdm_status tdm_solve_batched_noalloc(const tdm_handle* hs, int count, const float* const* F,
                                                const int64_t* ldF, double* const* X, const int64_t* ldX,
                                                const int64_t* N, void* stream) {
  if (count < 0 || (count > 0 && (!hs || !F || !ldF || !X || !ldX || !N))) return TDM_ERR_INVALID_ARG;
  if (count == 0) return TDM_OK;
  for (int k = 0; k < count; k++) {
    const tdm_status st = tdm_validate_solve(hs[k], F[k], ldF[k], X[k], ldX[k], N[k], TDM_FP32_REFINED);
    if (st != TDM_OK) return st;
    if (hs[k]->device != hs[0]->device || hs[k]->t != hs[0]->t) return TDM_ERR_INVALID_ARG;
  }
  // Not capturable: a captured copy from g_stage would re-read the host array
  // at every replay, after later calls have refilled it.  Refused before
  // anything is staged or enqueued.
  {
    CurrentDevice guard(hs[0]->device);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
      (void)cudaGetLastError();
      return TDM_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return TDM_ERR_NOT_IMPLEMENTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);

  // the work list's size, checked against the array before anything is enqueued
  int ne = 0;
  int64_t total = 0;
  for (int k = 0; k < count; k++) {
    if (N[k] == 0) continue;
    Entry e;
    e.k = k;
    e.t = hs[k]->t;
    if (ldF[k] > kRefMaxLd || ldX[k] > kRefMaxLd) return TDM_ERR_NOT_IMPLEMENTED;
    if (!tdm_refined_shape(hs[k]->M, e.t, hs[k]->tile_rhs, e.sh)) return TDM_ERR_NOT_IMPLEMENTED;
    const int64_t tiles = (N[k] + e.sh.R - 1) / e.sh.R;
    total += tiles;
    if (total > kMaxTiles) return TDM_ERR_TOO_LARGE;
    e.tiles = (int)tiles;
    e.cost = (double)hs[k]->n * (double)N[k];
    g_entries[ne++] = e;
  }
  if (ne == 0) return TDM_OK;

  // group by tile shape, biggest series first inside a group (series number
  // breaks ties, so the order is total and std::sort needs no buffer)
  std::sort(g_entries, g_entries + ne, [](const Entry& x, const Entry& y) {
    if (x.t != y.t) return x.t < y.t;
    if (x.sh.C != y.sh.C) return x.sh.C > y.sh.C;
    if (x.sh.R != y.sh.R) return x.sh.R > y.sh.R;
    if (x.sh.m != y.sh.m) return x.sh.m > y.sh.m;
    if (x.cost != y.cost) return x.cost > y.cost;
    return x.k < y.k;
  });
  int nitems = 0;
  for (int i = 0; i < ne; i++) {
    const Entry& e = g_entries[i];
    RefItem base = tdm_refined_item(hs[e.k], F[e.k], ldF[e.k], X[e.k], ldX[e.k], N[e.k], e.k, e.sh);
    for (int tile = 0; tile < e.tiles; tile++) {
      base.tile = tile;
      g_stage[nitems++] = base;
    }
  }

  CurrentDevice guard(hs[0]->device);
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();   // report only errors of this call
  RefItem* d_tiles = nullptr;
  tdm_status st = device_tiles(hs[0]->device, &d_tiles);
  if (st != TDM_OK) return st;
  // From pageable host memory: the call returns once g_stage has been copied
  // out, so the next call may refill it; the device copy is stream-ordered
  // after this stream's earlier launches that read g_tiles.  The driver may
  // stage such a copy synchronously: the call can then block the host until
  // the stream's earlier work has finished.
  TDM_CUDA_TRY(cudaMemcpyAsync(d_tiles, g_stage, sizeof(RefItem) * (size_t)nitems, cudaMemcpyHostToDevice, s));
  for (int i = 0; i < ne;) {
    int j = i, off = 0;
    for (int q = 0; q < i; q++) off += g_entries[q].tiles;
    int cnt = 0;
    while (j < ne && same_shape(g_entries[i], g_entries[j])) cnt += g_entries[j++].tiles;
    st = tdm_refined_launch(g_entries[i].sh, g_entries[i].t, d_tiles + off, nullptr, cnt, hs[0]->dev_err, s);
    if (st != TDM_OK) return st;
    i = j;
  }
  for (int k = 0; k < count; k++) TDM_CUDA_TRY(cudaEventRecord(hs[k]->last, s));
  return TDM_OK;
}
