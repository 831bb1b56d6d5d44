// tdm_large.cu -- systems larger than one thread-block cluster holds.
//
// The dichotomy applied one level up (Lemma 1 with separators between
// super-blocks; the reduced system of the separator values).  The rows are
// cut into K segments of at most L = 1024 t rows, separated by single rows
// q_1 < ... < q_{K-1}:
//   1. every segment's interior is a Dirichlet subproblem: y_j = A_j^-1 F_j,
//      solved by the segment's own plan (the cluster kernels), written straight
//      into X's rows;
//   2. x_i = y_i + phiL_j(i) x(q_{j-1}) + phiR_j(i) x(q_j) on segment j, with
//      phiL_j = A_j^-1 (-a e_first), phiR_j = A_j^-1 (-a e_last) formed at
//      prepare by the same plans;
//   3. substituting 2 into the rows q_j gives a symmetric tridiagonal system
//      for the separator values,
//         (b_q + a_{q-1} phiR_j(last) + a_q phiL_{j+1}(first)) x(q_j)
//           + a_{q-1} phiL_j(last) x(q_{j-1}) + a_q phiR_{j+1}(first) x(q_{j+1})
//           = F_q - a_{q-1} y_j(last) - a_q y_{j+1}(first),
//      solved by a plan of its own (in binary64 for the binary64 and the
//      refined solves, in binary32 for the binary32 solve);
//   4. one pass over X adds the separator terms of 2 and stores x(q_j).
// F is read once; X is written by the segment solves, then read and written
// once more by step 4.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tdm_internal.cuh"

namespace {

// unit right-hand sides of the homogeneous responses: column 0 = -a_{s-1} e_0
// (left separator), column 1 = -a_{s+m-1} e_{m-1} (right separator)
__global__ void k_unit_rhs(const double* __restrict__ a, int64_t s, int64_t m, bool left, bool right,
                           double* __restrict__ E) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    E[2 * i] = (left && i == 0) ? -a[s - 1] : 0.0;
    E[2 * i + 1] = (right && i == m - 1) ? -a[s + m - 1] : 0.0;
  }
}

// the reduced matrix: red_b[j] for separator j, red_a[j] between separators j and j+1
__global__ void k_reduced_matrix(const double* __restrict__ a, const double* __restrict__ b,
                                 const int64_t* __restrict__ seg, int K, const double* __restrict__ phi,
                                 double* __restrict__ red_a, double* __restrict__ red_b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K - 1) return;
  const int64_t q = seg[j + 1] - 1;                // separator row between segments j and j+1
  const int64_t last = q - 1, first = q + 1;       // neighbouring segment rows
  red_b[j] = b[q] + a[q - 1] * phi[2 * last + 1] + a[q] * phi[2 * first + 0];
  if (j + 1 < K - 1) {
    const int64_t q2 = seg[j + 2] - 1;             // next separator
    red_a[j] = a[q2 - 1] * phi[2 * (q2 - 1) + 0];   // row q2's coefficient of x(q)
  }
}

template <typename TF, typename TX, typename TR>
__global__ void k_reduced_rhs(const double* __restrict__ a, const int64_t* __restrict__ seg, int K,
                              const TF* __restrict__ F, int64_t ldF, const TX* __restrict__ X, int64_t ldX,
                              int64_t N, TR* __restrict__ R) {
  const int64_t total = (int64_t)(K - 1) * N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / N, c = k % N;
    const int64_t q = seg[j + 1] - 1;
    const double r = (double)F[q * ldF + c] - a[q - 1] * (double)X[(q - 1) * ldX + c] -
                     a[q] * (double)X[(q + 1) * ldX + c];
    R[j * N + c] = (TR)r;
  }
}

// X's arithmetic type throughout: binary32 X is combined in binary32 (the
// binary64 pipe runs at 1/64 of the binary32 rate on GB300), binary64 X in
// binary64
template <typename TX>
__global__ void k_combine(const int64_t* __restrict__ seg, int K, int64_t n, const double* __restrict__ phi,
                          const TX* __restrict__ Xs, int64_t N, TX* __restrict__ X, int64_t ldX) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    // segment of row i (K is small: a linear scan of the boundaries)
    int j = 0;
    while (j + 1 < K && i >= seg[j + 1]) j++;
    const bool sep = (j + 1 < K) && (i == seg[j + 1] - 1);
    const TX pl = (TX)((j > 0 && !sep) ? phi[2 * i] : 0.0);
    const TX pr = (TX)((j + 1 < K && !sep) ? phi[2 * i + 1] : 0.0);
    const TX* xl = Xs + (int64_t)(j > 0 ? j - 1 : 0) * N;
    const TX* xr = Xs + (int64_t)j * N;
    TX* row = X + i * ldX;
    for (int64_t c = threadIdx.x; c < N; c += blockDim.x) {
      if (sep) {
        row[c] = xr[c];
      } else {
        TX x = row[c];
        if (j > 0) x = fma(pl, xl[c], x);
        if (j + 1 < K) x = fma(pr, xr[c], x);
        row[c] = x;
      }
    }
  }
}

int grid_for(int64_t work) {
  const int64_t g = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

}  // namespace

// Builds the two-level structure of a symmetric plan p (prepared already) whose
// rows exceed L.  a and b are the caller's device arrays.
tdm_status tdm_prepare_large(tdm_plan_s* p, const double* a, const double* b, const tdm_options* opt,
                             cudaStream_t s) {
  const int64_t n = p->n, L = (int64_t)1024 * p->t;
  const int K = (int)((n + 1 + L) / (L + 1));   // segments of at most L rows, K - 1 separator rows
  const int64_t interior = n - (K - 1);
  std::vector<int64_t> seg(K + 1);              // segment j: rows [seg[j], seg[j+1] - 1), separator seg[j+1] - 1
  int64_t r = 0;
  for (int j = 0; j < K; j++) {
    const int64_t m = interior / K + (j < interior % K ? 1 : 0);
    seg[j] = r;
    r += m + (j + 1 < K ? 1 : 0);
  }
  seg[K] = n + 1;                                // so that seg[K] - 1 = n (no separator after the last)
  p->nseg = K;
  p->seg_host = new int64_t[K + 1];
  memcpy(p->seg_host, seg.data(), sizeof(int64_t) * (K + 1));
  p->subs = new tdm_plan_s*[K];
  for (int j = 0; j < K; j++) p->subs[j] = nullptr;
  TDM_CUDA_TRY(cudaMalloc(&p->seg_dev, sizeof(int64_t) * (K + 1)));
  TDM_CUDA_TRY(cudaMalloc(&p->phi, sizeof(double) * 2 * n));
  TDM_CUDA_TRY(cudaMemcpyAsync(p->seg_dev, seg.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, s));
  TDM_CUDA_TRY(cudaMemsetAsync(p->phi, 0, sizeof(double) * 2 * n, s));
  tdm_options o = opt ? *opt : tdm_options{0, 0, 0, 0};
  o.block_rows = p->t;
  for (int j = 0; j < K; j++) {
    const int64_t s0 = seg[j];
    const int64_t m = (j + 1 < K ? seg[j + 1] - 1 : n) - s0;
    tdm_handle h = nullptr;
    tdm_status st = tdm_prepare(m > 1 ? a + s0 : nullptr, b + s0, m, &o, s, &h);
    if (st != TDM_OK) return st;
    p->subs[j] = h;
    // homogeneous responses of the segment
    k_unit_rhs<<<grid_for(m), 256, 0, s>>>(a, s0, m, j > 0, j + 1 < K, p->phi + 2 * s0);
    TDM_CUDA_TRY(cudaGetLastError());
    double* E = nullptr;
    TDM_CUDA_TRY(cudaMalloc(&E, sizeof(double) * 2 * m));
    TDM_CUDA_TRY(cudaMemcpyAsync(E, p->phi + 2 * s0, sizeof(double) * 2 * m, cudaMemcpyDeviceToDevice, s));
    st = tdm_launch_solve(h, E, 2, p->phi + 2 * s0, 2, 2, TDM_FP64, s);
    cudaStreamSynchronize(s);
    cudaFree(E);
    if (st != TDM_OK) return st;
  }
  if (K > 1) {
    double *ra = nullptr, *rb = nullptr;
    TDM_CUDA_TRY(cudaMalloc(&ra, sizeof(double) * std::max(K - 2, 1)));
    TDM_CUDA_TRY(cudaMalloc(&rb, sizeof(double) * (K - 1)));
    k_reduced_matrix<<<(K + 127) / 128, 128, 0, s>>>(a, b, p->seg_dev, K, p->phi, ra, rb);
    tdm_status st = TDM_OK;
    if (cudaGetLastError() != cudaSuccess) st = TDM_ERR_CUDA;
    tdm_options ro{0, 1, 0, 0};   // no calibration: the reduced system is never solved refined
    tdm_handle h = nullptr;
    if (st == TDM_OK) st = tdm_prepare(K - 1 > 1 ? ra : nullptr, rb, K - 1, &ro, s, &h);
    cudaStreamSynchronize(s);
    cudaFree(ra);
    cudaFree(rb);
    if (st != TDM_OK) return st;
    p->reduced = h;
  }
  TDM_CUDA_TRY(cudaStreamSynchronize(s));
  return TDM_OK;
}

void tdm_free_large(tdm_plan_s* p) {
  if (p->subs) {
    for (int j = 0; j < p->nseg; j++)
      if (p->subs[j]) tdm_destroy(p->subs[j]);
    delete[] p->subs;
  }
  if (p->reduced) tdm_destroy(p->reduced);
  delete[] p->seg_host;
  cudaFree(p->seg_dev);
  cudaFree(p->phi);
}

tdm_status tdm_launch_large(tdm_plan_s* p, const void* F, int64_t ldF, void* X, int64_t ldX, int64_t N,
                            tdm_precision prec, cudaStream_t s) {
  const int K = p->nseg;
  const int64_t n = p->n;
  const size_t ei = prec == TDM_FP64 ? 8 : 4, eo = prec == TDM_FP32 ? 4 : 8;
  // 1. the segments' Dirichlet subproblems, straight into X's rows
  for (int j = 0; j < K; j++) {
    const int64_t s0 = p->seg_host[j];
    const tdm_status st = tdm_launch_solve(p->subs[j], static_cast<const char*>(F) + (size_t)s0 * ldF * ei, ldF,
                                           static_cast<char*>(X) + (size_t)s0 * ldX * eo, ldX, N, prec, s);
    if (st != TDM_OK) return st;
  }
  if (K == 1) return TDM_OK;
  // 2-3. the reduced system of the separator values (binary64 unless the solve is binary32)
  const bool red32 = prec == TDM_FP32;
  const size_t er = red32 ? 4 : 8;
  void *R = nullptr, *Xs = nullptr;
  TDM_CUDA_TRY(cudaMallocAsync(&R, er * (size_t)(K - 1) * N, s));
  TDM_CUDA_TRY(cudaMallocAsync(&Xs, er * (size_t)(K - 1) * N, s));
  const int g = grid_for((int64_t)(K - 1) * N);
  const double* a = p->a64;
  if (prec == TDM_FP64)
    k_reduced_rhs<double, double, double><<<g, 256, 0, s>>>(a, p->seg_dev, K, static_cast<const double*>(F), ldF,
                                                             static_cast<const double*>(X), ldX, N, static_cast<double*>(R));
  else if (prec == TDM_FP32)
    k_reduced_rhs<float, float, float><<<g, 256, 0, s>>>(a, p->seg_dev, K, static_cast<const float*>(F), ldF,
                                                          static_cast<const float*>(X), ldX, N, static_cast<float*>(R));
  else
    k_reduced_rhs<float, double, double><<<g, 256, 0, s>>>(a, p->seg_dev, K, static_cast<const float*>(F), ldF,
                                                            static_cast<const double*>(X), ldX, N, static_cast<double*>(R));
  TDM_CUDA_TRY(cudaGetLastError());
  tdm_status st = tdm_launch_solve(p->reduced, R, N, Xs, N, N, red32 ? TDM_FP32 : TDM_FP64, s);
  // 4. the separator terms and values
  if (st == TDM_OK) {
    const int gc = (int)std::min<int64_t>(n, 8192);
    if (prec == TDM_FP32)
      k_combine<float><<<gc, 256, 0, s>>>(p->seg_dev, K, n, p->phi, static_cast<const float*>(Xs), N,
                                          static_cast<float*>(X), ldX);
    else
      k_combine<double><<<gc, 256, 0, s>>>(p->seg_dev, K, n, p->phi, static_cast<const double*>(Xs), N,
                                           static_cast<double*>(X), ldX);
    if (cudaGetLastError() != cudaSuccess) st = TDM_ERR_CUDA;
  }
  cudaFreeAsync(R, s);
  cudaFreeAsync(Xs, s);
  return st;
}
