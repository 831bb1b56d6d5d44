// tdm_host.cu -- tdm_solve_host: the solve of a series whose right-hand sides
// and solutions live in host memory.  The columns are cut into chunks; each
// chunk is copied in, solved and copied out on three streams with two device
// staging buffers per direction, so that the copy of chunk k+1 in, the solve
// of chunk k and the copy of chunk k-1 out overlap.  With pinned host memory
// the time approaches that of the slowest of the three.
//
// Chunk width: on GB300 with pinned memory (n = 16384, N = 8192, refined) a
// step took 10.3 ms with chunks of 1024 columns, 7.2 ms with 2048, 8.1 ms with
// 4096 and 10.7 ms unchunked; the copies out (8 KB rows and narrower) run
// slower than contiguous ones.  Letting the solve kernel read F and write X in
// mapped host memory directly took 16.9 ms.
//
// Staging: the plan keeps two F and two X chunk buffers on the device, sized
// on first use for the largest chunk seen, and the two copy streams with
// their events; tdm_destroy frees them.  One copy per chunk and direction
// (cudaMemcpy2DAsync over the chunk's rows).
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "tdm_internal.cuh"

namespace {

struct HostStage {
  void* F[2] = {nullptr, nullptr};
  void* X[2] = {nullptr, nullptr};
  size_t bytesF = 0, bytesX = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t in_done[2] = {nullptr, nullptr};    // chunk k's F staged
  cudaEvent_t solved[2] = {nullptr, nullptr};     // chunk k solved (F buffer free, X ready)
  cudaEvent_t out_done[2] = {nullptr, nullptr};   // chunk k copied out (X buffer free)
  std::mutex mu;
};

size_t in_size(tdm_precision p) { return p == TDM_FP64 ? 8 : 4; }
size_t out_size(tdm_precision p) { return p == TDM_FP32 ? 4 : 8; }

tdm_status ensure(HostStage& st, size_t bF, size_t bX) {
  if (!st.h2d) {
    TDM_CUDA_TRY(cudaStreamCreateWithFlags(&st.h2d, cudaStreamNonBlocking));
    TDM_CUDA_TRY(cudaStreamCreateWithFlags(&st.d2h, cudaStreamNonBlocking));
    TDM_CUDA_TRY(cudaEventCreateWithFlags(&st.start, cudaEventDisableTiming));
    for (int i = 0; i < 2; i++) {
      TDM_CUDA_TRY(cudaEventCreateWithFlags(&st.in_done[i], cudaEventDisableTiming));
      TDM_CUDA_TRY(cudaEventCreateWithFlags(&st.solved[i], cudaEventDisableTiming));
      TDM_CUDA_TRY(cudaEventCreateWithFlags(&st.out_done[i], cudaEventDisableTiming));
    }
  }
  if (bF > st.bytesF || bX > st.bytesX) {
    // no copy of an earlier call may still use the old buffers
    TDM_CUDA_TRY(cudaStreamSynchronize(st.h2d));
    TDM_CUDA_TRY(cudaStreamSynchronize(st.d2h));
    for (int i = 0; i < 2; i++) {
      TDM_CUDA_TRY(cudaEventSynchronize(st.solved[i]));
      cudaFree(st.F[i]);
      cudaFree(st.X[i]);
      st.F[i] = st.X[i] = nullptr;
    }
    st.bytesF = st.bytesX = 0;
    for (int i = 0; i < 2; i++) {
      if (cudaMalloc(&st.F[i], bF) != cudaSuccess || cudaMalloc(&st.X[i], bX) != cudaSuccess) {
        (void)cudaGetLastError();
        return TDM_ERR_NO_MEMORY;
      }
    }
    st.bytesF = bF;
    st.bytesX = bX;
  }
  return TDM_OK;
}

}  // namespace

void tdm_host_stage_free(void* p) {
  HostStage* st = static_cast<HostStage*>(p);
  if (!st) return;
  for (int i = 0; i < 2; i++) {
    cudaFree(st->F[i]);
    cudaFree(st->X[i]);
    if (st->in_done[i]) cudaEventDestroy(st->in_done[i]);
    if (st->solved[i]) cudaEventDestroy(st->solved[i]);
    if (st->out_done[i]) cudaEventDestroy(st->out_done[i]);
  }
  if (st->start) cudaEventDestroy(st->start);
  if (st->h2d) cudaStreamDestroy(st->h2d);
  if (st->d2h) cudaStreamDestroy(st->d2h);
  delete st;
}

extern "C" tdm_status tdm_solve_host(tdm_handle h, const void* F, int64_t ldF, void* X, int64_t ldX, int64_t N,
                                     int64_t chunk, tdm_precision prec, void* stream) {
  if (!h || chunk < 0 || N < 0 || N > (int64_t(1) << 40)) return TDM_ERR_INVALID_ARG;
  if (prec != TDM_FP64 && prec != TDM_FP32 && prec != TDM_FP32_REFINED) return TDM_ERR_INVALID_ARG;
  if (h->general && prec == TDM_FP32_REFINED) return TDM_ERR_NOT_IMPLEMENTED;
  if (N == 0) return TDM_OK;
  if (!F || !X || ldF < N || ldX < N) return TDM_ERR_INVALID_ARG;
  const int64_t n = h->n;
  {   // F and X must not overlap
    const uintptr_t f0 = reinterpret_cast<uintptr_t>(F), x0 = reinterpret_cast<uintptr_t>(X);
    const uintptr_t f1 = f0 + ((size_t)(n - 1) * (size_t)ldF + (size_t)N) * in_size(prec);
    const uintptr_t x1 = x0 + ((size_t)(n - 1) * (size_t)ldX + (size_t)N) * out_size(prec);
    if (f0 < x1 && x0 < f1) return TDM_ERR_INVALID_ARG;
  }
  // chunk width: a multiple of 16 columns; by default about N / 4, at least 2048
  int64_t w = chunk > 0 ? chunk : std::max<int64_t>(2048, (N + 3) / 4);
  w = std::min<int64_t>(((w + 15) / 16) * 16, ((N + 15) / 16) * 16);
  const int64_t nchunks = (N + w - 1) / w;
  const size_t ei = in_size(prec), eo = out_size(prec);

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  struct Restore {
    int d;
    ~Restore() { if (d >= 0) cudaSetDevice(d); }
  } restore{prev != h->device ? prev : -1};
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  {   // host copies on helper streams do not belong in a graph capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TDM_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return TDM_ERR_NOT_IMPLEMENTED;
  }

  if (!h->host_stage) h->host_stage = new HostStage();
  HostStage& st = *static_cast<HostStage*>(h->host_stage);
  std::lock_guard<std::mutex> lock(st.mu);
  tdm_status rc = ensure(st, (size_t)n * (size_t)w * ei, (size_t)n * (size_t)w * eo);
  if (rc != TDM_OK) return rc;

  // nothing starts before the work already on the caller's stream
  TDM_CUDA_TRY(cudaEventRecord(st.start, s));
  TDM_CUDA_TRY(cudaStreamWaitEvent(st.h2d, st.start, 0));
  TDM_CUDA_TRY(cudaStreamWaitEvent(st.d2h, st.start, 0));
  for (int64_t k = 0; k < nchunks; k++) {
    const int b = (int)(k & 1);
    const int64_t c0 = k * w, cols = std::min<int64_t>(w, N - c0);
    // in: F buffer b is free once its last solve (chunk k-2, or an earlier call's) is done;
    // an event never recorded counts as complete
    TDM_CUDA_TRY(cudaStreamWaitEvent(st.h2d, st.solved[b], 0));
    TDM_CUDA_TRY(cudaMemcpy2DAsync(st.F[b], (size_t)w * ei, static_cast<const char*>(F) + (size_t)c0 * ei,
                                   (size_t)ldF * ei, (size_t)cols * ei, (size_t)n, cudaMemcpyHostToDevice, st.h2d));
    TDM_CUDA_TRY(cudaEventRecord(st.in_done[b], st.h2d));
    // solve: needs chunk k staged and X buffer b copied out (chunk k-2)
    TDM_CUDA_TRY(cudaStreamWaitEvent(s, st.in_done[b], 0));
    TDM_CUDA_TRY(cudaStreamWaitEvent(s, st.out_done[b], 0));
    rc = tdm_launch_solve(h, st.F[b], w, st.X[b], w, cols, prec, s);
    if (rc != TDM_OK) return rc;
    TDM_CUDA_TRY(cudaEventRecord(st.solved[b], s));
    // out
    TDM_CUDA_TRY(cudaStreamWaitEvent(st.d2h, st.solved[b], 0));
    TDM_CUDA_TRY(cudaMemcpy2DAsync(static_cast<char*>(X) + (size_t)c0 * eo, (size_t)ldX * eo, st.X[b],
                                   (size_t)w * eo, (size_t)cols * eo, (size_t)n, cudaMemcpyDeviceToHost, st.d2h));
    TDM_CUDA_TRY(cudaEventRecord(st.out_done[b], st.d2h));
  }
  // the caller's stream completes only after the last copies out
  for (int64_t k = std::max<int64_t>(0, nchunks - 2); k < nchunks; k++)
    TDM_CUDA_TRY(cudaStreamWaitEvent(s, st.out_done[k & 1], 0));
  TDM_CUDA_TRY(cudaEventRecord(h->last, s));
  return TDM_OK;
}
