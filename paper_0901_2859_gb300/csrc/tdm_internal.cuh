// tdm_internal.cuh -- plan layout and device helpers shared by the library's
// translation units (prepare, solve, backward, C ABI).  Not a public header.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tdm.h"

// ---------------------------------------------------------------------------
// Per-row coefficients of the solve step, [n][8] in the solve's arithmetic type.
// Rows are cut into blocks of t rows: block b = rows [b*t, min(b*t+t, n)).
// Block b >= 1 starts with separator row p_b = b*t; its interior is the rest.
// ---------------------------------------------------------------------------
enum {
  // first 4-vector: read by the forward pass (A2 + A3)
  kGR = 0,    // G_{p_{b+1}}(i): inverse row of the block's right separator (eq. beta_symn)
  kGL = 1,    // G_{p_b}(i): inverse row of the block's left separator
  kLF = 2,    // forward multiplier of the interior's local sweep (0 on the first interior row)
  // second 4-vector: read by the backward pass (A5)
  kC = 4,     // off-diagonal used by back substitution (0 on the last interior row)
  kINVD = 5,  // 1 / pivot of the local sweep (0 on a separator row)
  kPHIL = 6,  // interior response to a unit left separator value (1 on the separator row)
  kPHIR = 7,  // interior response to a unit right separator value
  kNCOEF = 8
};

// Residual coefficients of the refined path, [n][8] binary32:
// sigma_i = b_i + a_{i-1} + a_i (row sum) and a_i, each split into three
// binary32 parts whose sum equals the binary64 value (to 2^-72 relative).
// The first 4-vector holds the two leading parts of both (one vector load).
enum { kS0 = 0, kS1 = 1, kA0 = 2, kA1 = 3, kS2 = 4, kA2 = 5, kNRES = 8 };

// Device status bits written by the prepare kernels.
enum {
  kStatSingular = 1,      // zero or tiny pivot, vanishing inverse-row diagonal
  kStatNotDominant = 2,   // some row violates |b_i| >= |a_{i-1}| + |a_i|
  kStatStrict = 4,        // some row satisfies it strictly
  kStatNonFinite = 8,
  kStatNotSymmetrizable = 16   // tdm_prepare_general: some sub[k] * sup[k] <= 0 or not finite
};

struct tdm_plan_s {
  int64_t n = 0;
  int t = 0;               // rows per block
  int M = 0;               // number of blocks, M - 1 separators
  int refine_steps = 0;      // -1: tested per tile (cap 4); k > 0: exactly k corrections
  float contraction = 1.f;   // per-tile test: error after one correction ~ its size x this (1: untested)
  int tile_rhs = 0;          // right-hand sides per refined tile (0: by the shape rule)
  int general = 0;           // 1: a nonsymmetric matrix, symmetrized (tdm_prepare_general)
  int dominant = 0;
  double max_abs_z = 0.0;
  double min_abs_pivot = 0.0;
  int device = 0;
  // device buffers (owned)
  double* coef64 = nullptr;   // [n][8]
  float* coef32 = nullptr;    // [n][8]
  float* res32 = nullptr;     // [n][8]
  float* rtab = nullptr;      // [M + 1][kRefTabStride(t)] coefficient table of the refined kernel (tdm_refine.cuh)
  double* rR = nullptr;       // [M + 2]: rR[q] = Z^R_{p_q}(p_{q+1}), q = 1..M-2, else 0
  double* rL = nullptr;       // [M + 2]: rL[q] = Z^L_{p_q}(p_{q-1}), q = 2..M-1, else 0
  double* a64 = nullptr;      // [max(n-1,1)] copy of a (general plans: the symmetrized off-diagonal)
  double* tr = nullptr;       // [max(n-1,1)] general plans: t_{k+1} / t_k of the similarity T
  double* b64 = nullptr;      // [n] copy of b
  double* piv = nullptr;      // [4n] forward and backward pivots of A (double-double)
  unsigned long long* stat = nullptr;  // [8] device status / reductions
  int* dev_err = nullptr;     // [1] device error word of solves
  // cooperative refined launches (tdm_refine.cu): CTAs of the grid, their
  // scratch blocks and the groups' barrier counters
  int coop_grid = 0;
  float* coop_scr = nullptr;
  unsigned* coop_ctr = nullptr;
  // the same for the plain binary64 solve (tdm_solve.cu)
  int coop64_grid = 0;
  double* coop64_scr = nullptr;
  unsigned* coop64_ctr = nullptr;
  cudaEvent_t last = nullptr; // recorded after each solve
  void* host_stage = nullptr; // staging buffers and streams of tdm_solve_host (created on first use)
  // two levels (n beyond one cluster, tdm_large.cu): segments, their plans, responses, reduced plan
  int nseg = 0;
  int64_t* seg_host = nullptr;     // [nseg + 1] segment starts (the separator after segment j is seg[j+1] - 1)
  int64_t* seg_dev = nullptr;
  double* phi = nullptr;           // [n][2] responses of every segment row to its left / right separator
  tdm_plan_s** subs = nullptr;     // [nseg] the segments' plans
  tdm_plan_s* reduced = nullptr;   // the separator values' plan (nseg - 1 rows)
};

void tdm_host_stage_free(void* stage);
tdm_status tdm_prepare_large(tdm_plan_s* p, const double* a, const double* b, const tdm_options* opt,
                             cudaStream_t s);
void tdm_free_large(tdm_plan_s* p);
tdm_status tdm_launch_large(tdm_plan_s* p, const void* F, int64_t ldF, void* X, int64_t ldX, int64_t N,
                            tdm_precision prec, cudaStream_t s);

#define TDM_CUDA_TRY(expr)                                      \
  do {                                                          \
    cudaError_t _e = (expr);                                    \
    if (_e != cudaSuccess) {                                    \
      (void)cudaGetLastError();                                 \
      return TDM_ERR_CUDA;                                      \
    }                                                           \
  } while (0)

static inline bool tdm_aligned(const void* p, uintptr_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// ---------------------------------------------------------------------------
// Exact binary32 <-> binary64 conversions on the integer pipe.  On GB300 the
// F2F conversion instructions run at the binary64 rate (~2 per clock per SM),
// 60x slower than integer logic, so the solve kernels move values between the
// two formats by rebuilding the bit patterns.  Zeros stay on that path too;
// subnormal, infinite and NaN inputs call the hardware conversion out of line
// (a call, so that the conversion is never issued as predicated code).
// ---------------------------------------------------------------------------
static __device__ __noinline__ double tdm_f2d_hw(float f) { return (double)f; }
static __device__ __noinline__ float tdm_d2f_hw(double d) { return (float)d; }

__device__ __forceinline__ double tdm_f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  if ((a - 0x00800000u) >= 0x7f000000u && a != 0u) return tdm_f2d_hw(f);   // subnormal, inf, NaN
  const uint32_t hi = a == 0u ? u : (u & 0x80000000u) | ((a >> 3) + 0x38000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// binary64 -> binary32, round to nearest even (values in the normal binary32
// range and zeros; everything else takes the hardware conversion).
__device__ __forceinline__ float tdm_d2f(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d);
  const uint32_t lo = (uint32_t)__double2loint(d);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e <= 896u || e >= 1151u) {
    if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return tdm_d2f_hw(d);
  }
  uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;
  uint32_t bits = (hi & 0x80000000u) | ((e - 896u) << 23) | m;
  const uint32_t up = (rem > 0x10000000u) || (rem == 0x10000000u && (m & 1u));
  bits += up;  // a carry out of the mantissa correctly bumps the exponent
  return __uint_as_float(bits);
}

template <typename T> __device__ __forceinline__ double tdm_to_f64(T v);
template <> __device__ __forceinline__ double tdm_to_f64<float>(float v) { return tdm_f2d(v); }
template <> __device__ __forceinline__ double tdm_to_f64<double>(double v) { return v; }
template <typename T> __device__ __forceinline__ T tdm_from_f64(double v);
template <> __device__ __forceinline__ float tdm_from_f64<float>(double v) { return tdm_d2f(v); }
template <> __device__ __forceinline__ double tdm_from_f64<double>(double v) { return v; }

// Host-side entry points implemented in the other translation units.
tdm_status tdm_launch_solve(tdm_plan_s* p, const void* F, int64_t ldF, void* X, int64_t ldX,
                            int64_t N, tdm_precision prec, cudaStream_t s);
tdm_status tdm_launch_backward_sums(tdm_plan_s* p, const void* W, const void* X, int64_t ld,
                                    int64_t N, double* da, double* db, tdm_precision prec,
                                    cudaStream_t s);
// the cooperative binary64 solve's grid for a plan of M blocks of t rows (0:
// clusters are as good), and the bytes of its scratch
int tdm_plain_coop_choice(int M, int t, size_t* scr_bytes);
void tdm_batched_forget(const tdm_plan_s* p);
tdm_status tdm_launch_batched(tdm_plan_s* const* ps, int count, const void* const* F,
                              const int64_t* ldF, void* const* X, const int64_t* ldX,
                              const int64_t* N, tdm_precision prec, cudaStream_t s);
