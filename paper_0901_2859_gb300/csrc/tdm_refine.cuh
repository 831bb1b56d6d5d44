// tdm_refine.cuh -- work items and the coefficient table of the refined
// persistent kernel (shared by the single-series and the batched launch paths,
// and by the prepare step that builds the table).
#pragma once

#include <stdint.h>

#include "tdm_internal.cuh"

// ---------------------------------------------------------------------------
// Coefficient table of the refined kernel, [M + 1][kRefTabStride(t)] binary32
// (the extra block is all zeros).  Per block:
//  * t/2 row pairs of kRefTP floats: the kernel holds a block's rows as pairs
//    (row j, row j + t/2), so these coefficients are stored as such pairs,
//      GR, GL     beta weights G_{p_{b+1}}(i), G_{p_b}(i)        (eq. beta_symn)
//      PLH, PRH   phiL, phiR rounded to binary32                  (Lemma 1)
//      PLL, PRL   phiL - PLH, phiR - PRH rounded to binary32 (the first solve's
//                 correction is formed with phi to ~2^-48)
//      S0, S1     sigma_i = b_i + a_{i-1} + a_i as a binary32 pair (residual)
//      A0, A1     a_i as a binary32 pair (residual);
//  * the local sweep, row by row: the forward multipliers of rows 0 .. t-1
//    (t floats, four per vector load), then the back substitution's
//    (off-diagonal, 1 / pivot) of rows t-1, t-2, ..., 0 (2t floats, two rows
//    per vector load, in the order the substitution walks them);
//  * 4 floats: A0, A1 of the row before the block (a_{row0-1}), 0, 0.
// Rows at or past n are zeros.
// ---------------------------------------------------------------------------
enum {
  kRT_GR = 0, kRT_GL = 2, kRT_PLH = 4, kRT_PRH = 6, kRT_PLL = 8, kRT_PRL = 10,
  kRT_S0 = 12, kRT_S1 = 14, kRT_A0 = 16, kRT_A1 = 18, kRefTP = 20
};
__host__ __device__ constexpr int kRefLF(int t) { return (t / 2) * kRefTP; }        // forward multipliers
__host__ __device__ constexpr int kRefCI(int t) { return kRefLF(t) + t; }            // back substitution
__host__ __device__ constexpr int kRefTail(int t) { return kRefCI(t) + 2 * t; }      // a_{row0-1}
__host__ __device__ constexpr int kRefTabStride(int t) { return kRefTail(t) + 4; }

// one tile of one series (an entry of a device-resident work list)
struct RefItem {
  const float* F;
  double* X;
  int64_t ldF, ldX;
  const float* tab;    // [M + 1][kRefTabStride(t)] coefficient table
  int m, g;            // blocks per CTA, CTAs of the group that solves the tile
  const double* rR;
  const double* rL;
  int n, M, N, tile;
  int series;          // series number: ratios are set up again when it changes
  int steps;           // corrections: k >= 1 exactly k; -1 tested per tile; -2 calibration
  float contraction;   // tested: estimated error after the first correction = its size x this
  int pad1;
};

// Grouped launches: a unit is one step of a cluster, in which every CTA works
// on the item units[u * kUnitW + rank] (a null item when it has nothing to
// do).  An item of group size g occupies the g CTAs of an aligned range
// (rank & ~(g - 1) .. + g - 1); g is a power of two.  Cluster k walks units
// ustart[k] .. ustart[k + 1] - 1 in order.
constexpr int kUnitW = 16;

// A run of a cooperative batched launch: tiles item0 .. item0 + ntiles - 1 (of
// one series) on the CTAs first .. first + g - 1; its barrier counter is the
// run's index.
struct RefRun {
  int item0, ntiles, first, g;
};

struct RefLaunch {
  const RefItem* items;   // work list (device); unused when single
  const int* units;       // grouped: [units][kUnitW] item of every CTA; runs: the run ids of every CTA, in order
  const int* ustart;      // grouped: [clusters + 1] first unit of every cluster; runs: [CTAs + 1] into units
  const RefRun* runs;     // runs: the runs
  RefItem one;            // the series of a single-series launch (item i = its tile i)
  int nitems;             // single: tiles; list: items (cluster k takes k, k + clusters, ...)
  int single;
  int m, C;               // single: blocks per CTA; CTAs per cluster (per group: cooperative)
  int* err;
  float* scr;             // cooperative: scratch blocks of the CTAs
  unsigned* ctr;          // cooperative: barrier counters of the groups (zero at launch)
};

// tile shape of the refined kernel for a series of M blocks of t rows
struct RefShape {
  int R = 0, NT = 0, m = 0, C = 0, threads = 0;
  bool sm_coef = true;   // coefficient table staged in shared memory
  size_t smem = 0;
};

// largest row stride (elements) of F and X the refined kernel addresses with
// 32-bit row offsets
constexpr int64_t kRefMaxLd = int64_t(1) << 26;

// steps value of a calibration solve: kRefineCalibSteps corrections, with the
// size of every correction recorded
constexpr int kRefineCalib = -2;
constexpr int kRefineCalibSteps = 4;

// pref: requested right-hand sides per tile (0 = by the rule)
bool tdm_refined_shape(int M, int t, int pref, RefShape& sh);
// enqueue one launch over `nitems` items (items == nullptr: single series `one`); every CTA of a
// cluster works on the same item (g = sh.C; list items carry their own m <= NT / R)
tdm_status tdm_refined_launch(const RefShape& sh, int t, const RefItem* items, const RefItem* one,
                              int nitems, int* err, cudaStream_t s);
// enqueue a grouped launch: `nclusters` clusters of sh.C CTAs walk the unit
// lists (sh.m is not used: every item carries its own m and g)
tdm_status tdm_refined_launch_grouped(const RefShape& sh, int t, const RefItem* items, const int* units,
                                      const int* ustart, int nclusters, int* err, cudaStream_t s);
// clusters of sh.C CTAs of the shape's kernel that the device holds at once
int tdm_refined_max_clusters(const RefShape& sh, int t);
// A cooperative launch over runs (sh: the kernel's shape; grid CTAs): CTA b
// walks the runs rlist[rstart[b]] .. rlist[rstart[b + 1] - 1]; the nruns
// counters ctr[32 * id] are zeroed on the stream first; scr holds grid
// scratch blocks (tdm_refined_coop_scratch).
int tdm_refined_coop_runs_grid(const RefShape& sh, int t);
tdm_status tdm_refined_launch_coop_runs(const RefShape& sh, int t, const RefItem* items, const RefRun* runs,
                                        const int* rlist, const int* rstart, int nruns, int grid, float* scr,
                                        unsigned* ctr, int* err, cudaStream_t s);
// Cooperative launches of one series (groups of sh.C consecutive CTAs in
// place of clusters): the largest grid of whole groups the device holds at
// once (0 if none), the bytes of scratch that grid needs, and the launch (its
// counters are zeroed on the stream first).
int tdm_refined_coop_grid(const RefShape& sh, int t);
// the cooperative grid when the rule prefers it to clusters for this shape, else 0
int tdm_refined_coop_choice(const RefShape& sh, int t);
size_t tdm_refined_coop_scratch(const RefShape& sh, int grid);
tdm_status tdm_refined_launch_coop(const RefShape& sh, int t, const RefItem& one, int ntiles, int* err, float* scr,
                                   unsigned* ctr, int grid, cudaStream_t s);
// the refined solve of one series (one single-series launch; cooperative when
// the plan chose it at prepare and allow_coop is set -- not for launches that
// run side by side with others, which a cooperative grid cannot share the GPU with)
tdm_status tdm_launch_refined(tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX, int64_t N,
                              cudaStream_t s, bool allow_coop = true);
// the calibration record: max over tiles of max|d_k| / max|x| for corrections
// k = 1 .. kRefineCalibSteps of calibration solves (cleared, or read into ratios)
tdm_status tdm_calibration_record(bool clear, float* ratios, cudaStream_t s);
// an item of series p in tile shape sh (every CTA of the cluster on it: m = sh.m, g = sh.C)
RefItem tdm_refined_item(const tdm_plan_s* p, const float* F, int64_t ldF, double* X, int64_t ldX,
                         int64_t N, int series, const RefShape& sh);
