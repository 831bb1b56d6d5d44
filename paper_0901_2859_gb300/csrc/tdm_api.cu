// tdm_api.cu -- the C ABI of include/tdm.h: argument validation, dispatch to
// the solve kernels, the backward row sums, batched solves, plan info.
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "tdm_internal.cuh"
#include "tdm_tma.cuh"
#include "tdm_iface_df.cuh"

tdm_status tdm_launch_plain(tdm_plan_s* p, const void* F, int64_t ldF, void* X, int64_t ldX,
                            int64_t N, bool fp64, cudaStream_t s);
tdm_status tdm_launch_refined(tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX,
                              int64_t N, cudaStream_t s, bool allow_coop);

namespace {

size_t elem_in(tdm_precision prec) { return prec == TDM_FP64 ? 8 : 4; }
size_t elem_out(tdm_precision prec) { return prec == TDM_FP32 ? 4 : 8; }

bool overlaps(const void* p0, size_t bytes0, const void* p1, size_t bytes1) {
  const uintptr_t a0 = (uintptr_t)p0, a1 = (uintptr_t)p1;
  return a0 < a1 + bytes1 && a1 < a0 + bytes0;
}

tdm_status validate_solve(const tdm_plan_s* h, const void* F, int64_t ldF, const void* X,
                          int64_t ldX, int64_t N, tdm_precision prec) {
  if (!h) return TDM_ERR_INVALID_ARG;
  if (prec != TDM_FP64 && prec != TDM_FP32 && prec != TDM_FP32_REFINED) return TDM_ERR_INVALID_ARG;
  // the refined residual is formed for a symmetric matrix (its edge fluxes are shared by both rows)
  if (h->general && prec == TDM_FP32_REFINED) return TDM_ERR_NOT_IMPLEMENTED;
  if (N < 0 || N > (int64_t(1) << 40)) return TDM_ERR_INVALID_ARG;
  if (N == 0) return TDM_OK;
  if (!F || !X || ldF < N || ldX < N) return TDM_ERR_INVALID_ARG;
  if (!tdm_aligned(F, 16) || !tdm_aligned(X, 16)) return TDM_ERR_INVALID_ARG;
  const size_t bf = ((size_t)(h->n - 1) * (size_t)ldF + (size_t)N) * elem_in(prec);
  const size_t bx = ((size_t)(h->n - 1) * (size_t)ldX + (size_t)N) * elem_out(prec);
  if (overlaps(F, bf, X, bx)) return TDM_ERR_INVALID_ARG;
  return TDM_OK;
}

// Records the plan's completion event, except while the stream is being
// captured into a CUDA graph (the graph's launches are synchronized by the
// caller; an event recorded inside a capture cannot be waited on afterwards).
cudaError_t record_last(tdm_plan_s* h, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return cudaSuccess;
  return cudaEventRecord(h->last, s);
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// Backward row sums, deterministic: one CTA per row, each thread sums a fixed
// strided subset of right-hand sides in order, then a fixed-shape tree.
template <typename T>
__global__ void __launch_bounds__(256) k_grad_rows(const T* __restrict__ L, const T* __restrict__ X,
                                                   int64_t ld, int64_t N, int64_t n,
                                                   double* __restrict__ da, double* __restrict__ db) {
  __shared__ double sa[256], sb[256];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    double accb = 0.0, acca = 0.0;
    const bool has_next = i + 1 < n;
    for (int64_t r = threadIdx.x; r < N; r += blockDim.x) {
      const double li = (double)L[i * ld + r], xi = (double)X[i * ld + r];
      accb = fma(li, xi, accb);
      if (has_next) {
        const double ln = (double)L[(i + 1) * ld + r], xn = (double)X[(i + 1) * ld + r];
        acca = fma(li, xn, acca);
        acca = fma(ln, xi, acca);
      }
    }
    sa[threadIdx.x] = acca;
    sb[threadIdx.x] = accb;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        sa[threadIdx.x] += sa[threadIdx.x + w];
        sb[threadIdx.x] += sb[threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (db) db[i] = -sb[0];
      if (da && has_next) da[i] = -sa[0];
    }
    __syncthreads();
  }
}

// The same sums for binary32 Lambda and X without binary64 arithmetic (one
// binary64 operation costs as much issue as 64 binary32 ones on GB300): each
// product is formed exactly as p + e (e = fma(l, x, -p)), added to a binary32
// pair accumulator by Knuth's TwoSum with the errors gathered in the low word
// (about 2^-44 relative to the sum of |terms| over a row of 2048 terms).  One
// warp per row: lane k sums the right-hand sides k, k + 32, ... in order, the
// lanes' pairs are added in a fixed butterfly, lane 0 rounds the pair to
// binary64.  Deterministic.
// (every operation an intrinsic with round-to-nearest, never contracted into
// an FMA, so that TwoSum's error term is exact)
__device__ __forceinline__ void acc_product(float l, float x, float& hi, float& lo) {
  const float p = __fmul_rn(l, x);
  const float e = fmaf(l, x, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}
__device__ __forceinline__ void add_pair(float& hi, float& lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, l2));
}
__global__ void __launch_bounds__(256) k_grad_rows_f32(const float* __restrict__ L, const float* __restrict__ X,
                                                       int64_t ld, int64_t N, int64_t n,
                                                       double* __restrict__ da, double* __restrict__ db) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const bool has_next = i + 1 < n;
    float bh = 0.f, bl = 0.f, ah = 0.f, al = 0.f;
    const float* Li = L + i * ld;
    const float* Xi = X + i * ld;
    for (int64_t r = lane; r < N; r += 32) {
      const float li = Li[r], xi = Xi[r];
      acc_product(li, xi, bh, bl);
      if (has_next) {
        acc_product(li, Xi[ld + r], ah, al);
        acc_product(Li[ld + r], xi, ah, al);
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const float bh2 = __shfl_xor_sync(0xffffffffu, bh, o), bl2 = __shfl_xor_sync(0xffffffffu, bl, o);
      const float ah2 = __shfl_xor_sync(0xffffffffu, ah, o), al2 = __shfl_xor_sync(0xffffffffu, al, o);
      add_pair(bh, bl, bh2, bl2);
      add_pair(ah, al, ah2, al2);
    }
    if (lane == 0) {
      if (db) db[i] = -((double)bh + (double)bl);
      if (da && has_next) da[i] = -((double)ah + (double)al);
    }
  }
}

// A wait on an mbarrier that no thread arrives at: the bounded wait of the
// solve kernels, with a caller-chosen limit, must give up and report.
__global__ void k_wait_selftest(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) tdm_mbar_init(&bar, 1);
  __syncthreads();
  (void)tdm_mbar_wait(&bar, 0u, err, limit);
}

}  // namespace

// The group barrier of the cooperative launches with a member that never
// arrives: CTA 1 of a group of two returns at once, CTA 0 arrives and waits,
// gives up after `limit` polls and records kDevErrGroupTimeout.
__global__ void k_group_selftest(unsigned* ctr, int* err, int limit) {
  if (blockIdx.x != 0) return;
  tdmk::Link<true> lk;
  lk.me = 0;
  lk.first = 0;
  lk.stride = 0;
  lk.g = 2;
  lk.ctr = ctr;
  lk.err = err;
  lk.spin_limit = limit;
  lk.arrive();
  lk.wait();
}

extern "C" tdm_status tdm_selftest_group_timeout(int64_t limit_polls, void* stream) {
  if (limit_polls < 1 || limit_polls > (int64_t(1) << 24)) return TDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  unsigned* d = nullptr;   // [0]: the counter, [32]: the error word
  TDM_CUDA_TRY(cudaMalloc(&d, 64 * sizeof(unsigned)));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, 64 * sizeof(unsigned), s);
  if (e == cudaSuccess) {
    int* err = reinterpret_cast<int*>(d + 32);
    int limit = (int)limit_polls;
    void* args[] = {&d, &err, &limit};
    e = cudaLaunchCooperativeKernel((void*)k_group_selftest, dim3(2), dim3(64), args, 0, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d + 32, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return TDM_ERR_CUDA;
  }
  return h == kDevErrGroupTimeout ? TDM_ERR_TIMEOUT : TDM_OK;
}

extern "C" tdm_status tdm_selftest_wait_timeout(int64_t limit_cycles, void* stream) {
  if (limit_cycles < 1 || limit_cycles > (int64_t(1) << 31)) return TDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  int* d = nullptr;
  TDM_CUDA_TRY(cudaMalloc(&d, sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(d, (long long)limit_cycles);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return TDM_ERR_CUDA;
  }
  return h == kDevErrTmaTimeout ? TDM_ERR_TIMEOUT : TDM_OK;
}

// argument checks of tdm_solve, for the entry points defined in other files
tdm_status tdm_validate_solve(const tdm_plan_s* h, const void* F, int64_t ldF, const void* X, int64_t ldX,
                              int64_t N, tdm_precision prec) {
  return validate_solve(h, F, ldF, X, ldX, N, prec);
}

tdm_status tdm_launch_solve(tdm_plan_s* p, const void* F, int64_t ldF, void* X, int64_t ldX,
                            int64_t N, tdm_precision prec, cudaStream_t s) {
  tdm_status st = TDM_ERR_INVALID_ARG;
  switch (prec) {
    case TDM_FP64: st = tdm_launch_plain(p, F, ldF, X, ldX, N, true, s); break;
    case TDM_FP32: st = tdm_launch_plain(p, F, ldF, X, ldX, N, false, s); break;
    case TDM_FP32_REFINED:
      st = tdm_launch_refined(p, static_cast<const float*>(F), ldF, static_cast<double*>(X), ldX, N, s, true);
      break;
  }
  // a plan beyond one cluster: the two-level solve (the direct kernels refuse before launching)
  if (st == TDM_ERR_NOT_IMPLEMENTED && p->nseg > 0) st = tdm_launch_large(p, F, ldF, X, ldX, N, prec, s);
  return st;
}

tdm_status tdm_launch_backward_sums(tdm_plan_s* p, const void* W, const void* X, int64_t ld,
                                    int64_t N, double* da, double* db, tdm_precision prec,
                                    cudaStream_t s) {
  (void)W;
  if (!da && !db) return TDM_OK;
  const int64_t n = p->n;
  int grid = n < 65536 ? (int)n : 65536;
  if (prec != TDM_FP32)   // Lambda and X in binary64 (the binary64 and the refined solves)
    k_grad_rows<double><<<grid, 256, 0, s>>>(static_cast<const double*>(W), static_cast<const double*>(X),
                                             ld, N, n, da, db);
  else   // binary32 pairs: one warp per row
    k_grad_rows_f32<<<(int)std::min<int64_t>((n + 7) / 8, 65536), 256, 0, s>>>(
        static_cast<const float*>(W), static_cast<const float*>(X), ld, N, n, da, db);
  TDM_CUDA_TRY(cudaGetLastError());
  return TDM_OK;
}

extern "C" tdm_status tdm_solve(tdm_handle h, const void* F, int64_t ldF, void* X, int64_t ldX,
                                int64_t N, tdm_precision prec, void* stream) {
  tdm_status st = validate_solve(h, F, ldF, X, ldX, N, prec);
  if (st != TDM_OK || N == 0) return st;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();   // report only errors of this call
  st = tdm_launch_solve(h, F, ldF, X, ldX, N, prec, s);
  if (st != TDM_OK) return st;
  TDM_CUDA_TRY(record_last(h, s));
  return TDM_OK;
}

extern "C" tdm_status tdm_solve_batched(const tdm_handle* hs, int count, const void* const* F,
                                        const int64_t* ldF, void* const* X, const int64_t* ldX,
                                        const int64_t* N, tdm_precision prec, void* stream) {
  if (count < 0 || (count > 0 && (!hs || !F || !ldF || !X || !ldX || !N))) return TDM_ERR_INVALID_ARG;
  if (count == 0) return TDM_OK;
  for (int k = 0; k < count; k++) {
    tdm_status st = validate_solve(hs[k], F[k], ldF[k], X[k], ldX[k], N[k], prec);
    if (st != TDM_OK) return st;
    if (hs[k]->device != hs[0]->device || hs[k]->t != hs[0]->t) return TDM_ERR_INVALID_ARG;
  }
  DeviceGuard g(hs[0]->device);
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  tdm_status st = tdm_launch_batched(const_cast<tdm_plan_s* const*>(hs), count, F, ldF, X, ldX, N, prec, s);
  if (st != TDM_OK) return st;
  for (int k = 0; k < count; k++) TDM_CUDA_TRY(record_last(hs[k], s));
  return TDM_OK;
}

extern "C" tdm_status tdm_solve_backward(tdm_handle h, const void* W, const void* X, int64_t ld,
                                         int64_t N, void* dF, double* da, double* db,
                                         tdm_precision prec, void* stream) {
  if (!h) return TDM_ERR_INVALID_ARG;
  if (prec != TDM_FP64 && prec != TDM_FP32 && prec != TDM_FP32_REFINED) return TDM_ERR_INVALID_ARG;
  if (h->general) return TDM_ERR_NOT_IMPLEMENTED;   // the adjoint of a nonsymmetric A is another matrix
  if (N < 0 || ld < N) return TDM_ERR_INVALID_ARG;
  if (N == 0) {
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (da && h->n > 1) TDM_CUDA_TRY(cudaMemsetAsync(da, 0, sizeof(double) * (h->n - 1), s));
    if (db) TDM_CUDA_TRY(cudaMemsetAsync(db, 0, sizeof(double) * h->n, s));
    return TDM_OK;
  }
  if (!W || !X || !dF) return TDM_ERR_INVALID_ARG;
  if (!tdm_aligned(X, 16) || (da && !tdm_aligned(da, 8)) || (db && !tdm_aligned(db, 8)))
    return TDM_ERR_INVALID_ARG;
  tdm_status st = validate_solve(h, W, ld, dF, ld, N, prec);
  if (st != TDM_OK) return st;
  const size_t bytes = ((size_t)(h->n - 1) * (size_t)ld + (size_t)N) * elem_out(prec);   // X and dF
  if (overlaps(X, bytes, dF, bytes)) return TDM_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  st = tdm_launch_solve(h, W, ld, dF, ld, N, prec, s);   // Lambda = A^{-1} W (A = A^T)
  if (st != TDM_OK) return st;
  st = tdm_launch_backward_sums(h, dF, X, ld, N, da, db, prec, s);
  if (st != TDM_OK) return st;
  TDM_CUDA_TRY(record_last(h, s));
  return TDM_OK;
}

extern "C" tdm_status tdm_get_info(tdm_handle h, tdm_info* info) {
  if (!h || !info) return TDM_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  (void)cudaGetLastError();
  TDM_CUDA_TRY(cudaEventSynchronize(h->last));
  int err = 0;
  TDM_CUDA_TRY(cudaMemcpy(&err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  memset(info, 0, sizeof(*info));
  info->n = h->n;
  info->block_rows = h->t;
  info->num_blocks = h->M;
  info->dominant = h->dominant;
  info->refine_steps = h->refine_steps;
  info->contraction = h->contraction;
  info->general = h->general;
  info->max_abs_z = h->max_abs_z;
  info->min_abs_pivot = h->min_abs_pivot;
  info->device_error = err;
  info->tile_rhs = h->tile_rhs;
  return TDM_OK;
}

extern "C" const char* tdm_status_string(tdm_status s) {
  switch (s) {
    case TDM_OK: return "TDM_OK";
    case TDM_ERR_INVALID_ARG: return "TDM_ERR_INVALID_ARG";
    case TDM_ERR_SINGULAR: return "TDM_ERR_SINGULAR";
    case TDM_ERR_CUDA: return "TDM_ERR_CUDA";
    case TDM_ERR_NO_MEMORY: return "TDM_ERR_NO_MEMORY";
    case TDM_ERR_NOT_CONVERGED: return "TDM_ERR_NOT_CONVERGED";
    case TDM_ERR_TIMEOUT: return "TDM_ERR_TIMEOUT";
    case TDM_ERR_NOT_IMPLEMENTED: return "TDM_ERR_NOT_IMPLEMENTED";
    case TDM_ERR_TOO_LARGE: return "TDM_ERR_TOO_LARGE";
  }
  return "TDM_ERR_UNKNOWN";
}
