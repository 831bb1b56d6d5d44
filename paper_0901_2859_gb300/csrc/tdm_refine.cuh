// tdm_refine.cuh -- work items of the refined persistent kernel (shared by the
// single-series and the batched launch paths).
#pragma once

#include <stdint.h>

#include "tdm_internal.cuh"

// one tile of one series (an entry of a device-resident work list)
struct RefItem {
  const float* F;
  double* X;
  int64_t ldF, ldX;
  const float* coef;   // [n][8] solve coefficients (binary32)
  const float* res;    // [n][8] residual coefficients
  const double* rR;
  const double* rL;
  int n, M, N, tile;
  int series;          // series number: ratios are set up again when it changes
  int steps;           // refinement steps (0 = adaptive)
  int pad0, pad1;
};

struct RefLaunch {
  const RefItem* items;   // work list (device); unused when single
  RefItem one;            // the series of a single-series launch (item i = its tile i)
  int nitems;
  int single;
  int m, C;               // blocks per CTA, CTAs per cluster
  int* err;
};

// tile shape of the refined kernel for a series of M blocks of t rows
struct RefShape {
  int R = 0, NT = 0, m = 0, C = 0, threads = 0;
  bool sm_coef = true;   // coefficient rows staged in shared memory
  size_t smem = 0;
};

// pref: requested right-hand sides per tile (0 = by the rule)
bool tdm_refined_shape(int M, int t, int pref, RefShape& sh);
// enqueue one launch over `nitems` items (items == nullptr: single series `one`)
tdm_status tdm_refined_launch(const RefShape& sh, int t, const RefItem* items, const RefItem* one,
                              int nitems, int* err, cudaStream_t s);
// the prepare-time calibration's view of the corrections per-tile-tested tiles made
tdm_status tdm_corrections_counter(bool clear, int* value, cudaStream_t s);
RefItem tdm_refined_item(const tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX,
                         int64_t N, int series);
