// tdm_batched.cu -- many matrices with their own right-hand sides (placeholder: one launch each).
#include "tdm_internal.cuh"

tdm_status tdm_launch_batched(tdm_plan_s* const* ps, int count, const void* const* F,
                              const int64_t* ldF, void* const* X, const int64_t* ldX,
                              const int64_t* N, tdm_precision prec, cudaStream_t s) {
  for (int k = 0; k < count; k++) {
    if (N[k] == 0) continue;
    tdm_status st = tdm_launch_solve(ps[k], F[k], ldF[k], X[k], ldX[k], N[k], prec, s);
    if (st != TDM_OK) return st;
  }
  return TDM_OK;
}
