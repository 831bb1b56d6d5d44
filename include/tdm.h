/*
 * tdm.h -- C ABI of the GB300 library for series of symmetric tridiagonal
 * systems solved by the parallel dichotomy (parallel sweep) method of
 * A. V. Terekhov, "Parallel dichotomy algorithm for solving tridiagonal SLAEs".
 *
 * Problem (Section 2, eq. main_eq3): A X_n = F_n, n = 1..N, one constant,
 * symmetric, nondegenerate tridiagonal A with diagonal b_0..b_{n-1} and
 * off-diagonal a_0..a_{n-2} (A[i][i+1] = A[i+1][i] = a_i).
 *
 * Method (Algorithms 3 and 4, Theorem 2, Lemma 1): the rows are cut into M
 * blocks of `block_rows` rows; block j >= 1 starts with a separator row.
 *   prepare  (Algorithm 3/4 step 1, once per matrix): inverse rows G_k at the
 *            separators over the two adjacent blocks (eq. green_v, Lemma 2),
 *            the homogeneous ratios Z^R_k(k'), Z^L_k(k') between neighbouring
 *            separators (eq. z_vector), the blocks' local sweep coefficients
 *            and their homogeneous solutions; all in binary64 on the GPU.
 *   solve    (step 2, per right-hand side): block-local dot products beta with
 *            the inverse rows (eq. beta_symn), separator values from Theorem 2
 *            evaluated as two first-order recurrences (in the arithmetic of
 *            the precision, see tdm_precision), then the block interiors from
 *            the local sweep plus a correction with the two separator values
 *            (Lemma 1).
 *
 * Conventions for every entry point
 *  - Pointers to matrix data (a, b, F, X, W, dF, da, db) are DEVICE pointers
 *    owned by the caller; the library never frees or keeps them.
 *  - Right-hand sides are row-major [n][ld] with the right-hand sides
 *    contiguous: element (row i, rhs r) is at F[i*ld + r]  (a PyTorch tensor
 *    of shape (n, N) with stride (ld, 1)).  ld >= N.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Solves are asynchronous: a return of TDM_OK means the work was
 *    validated and enqueued; device-side conditions are reported through
 *    tdm_get_info, which synchronizes on the plan's last solve.
 *  - Invalid arguments are rejected on the host before any launch with
 *    TDM_ERR_INVALID_ARG; nothing is enqueued in that case.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 *  - Refined and binary64 solves of one plan must be ordered on the device
 *    (one stream, or streams ordered by events): where clusters of the plan's
 *    width would leave many CTA slots idle (13 to 16 CTAs per tile), the solve
 *    is a cooperative launch whose CTA groups exchange values through a
 *    scratch buffer of the plan.
 *  - Solves may be captured into a CUDA graph.  A captured solve is not
 *    tracked by tdm_get_info / tdm_destroy; synchronize the graph's stream
 *    before destroying a plan it uses.  A batched call builds its device work
 *    list on first use of an argument set (not capturable): call it once with
 *    the same arguments before capturing it.
 */
#ifndef TDM_H
#define TDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdm_plan_s* tdm_handle;

typedef enum {
  TDM_OK = 0,
  TDM_ERR_INVALID_ARG = 1,      /* bad size, stride, pointer alignment, aliasing, null handle */
  TDM_ERR_SINGULAR = 2,         /* a binary64 pivot or an inverse-row diagonal vanished */
  TDM_ERR_CUDA = 3,             /* a CUDA call or kernel launch failed */
  TDM_ERR_NO_MEMORY = 4,        /* device allocation failed */
  TDM_ERR_NOT_CONVERGED = 5,    /* refinement did not reach its tolerance within its cap */
  TDM_ERR_TIMEOUT = 6,          /* a bounded device wait gave up */
  TDM_ERR_NOT_IMPLEMENTED = 7,  /* the requested combination is not available */
  TDM_ERR_TOO_LARGE = 8         /* the work exceeds a fixed capacity (tdm_solve_batched_noalloc) */
} tdm_status;

/* Arithmetic of a solve and the dtypes of F and X:
 *   TDM_FP64          F, X binary64; sweeps and dot products in binary64.
 *   TDM_FP32          F, X binary32; sweeps, dot products and the separator
 *                     recurrences (warp scans over products of the binary64
 *                     ratios, rounded to binary32) all in binary32.  Measured
 *                     relative error at n = 16384, a = -1, b = 2 + s:
 *                     4.3e-7 (s = 1e-6, condition ~4e6), 3.5e-7 (s = 1e-2).
 *   TDM_FP32_REFINED  F binary32, X binary64; binary32 solves corrected by
 *                     iterative refinement whose residual F - A X is formed
 *                     with error-free binary32 transformations (at least
 *                     binary64 accuracy), X accumulated as a binary32 pair. */
typedef enum { TDM_FP64 = 0, TDM_FP32 = 1, TDM_FP32_REFINED = 2 } tdm_precision;

typedef struct {
  int block_rows;    /* rows per block (the paper's subvector size); 0 = automatic (32).
                        Allowed: 16 or 32. */
  int refine_steps;  /* TDM_FP32_REFINED corrections:
                          k in 1..4: exactly k, no test;
                          -1: every tile of right-hand sides tests its own corrections: after
                              the first, stop if its size max|d_1| / max|x| times the plan's
                              contraction is below 4e-12; after the k-th (k >= 2), stop if the
                              estimated relative error max|d_k|^2 / (max|x| max|d_{k-1}|) is
                              below 1e-12; at most 4 (device_error 2 otherwise).  Requested
                              explicitly, the contraction is 1 (at least two corrections);
                          0 (automatic): -1 with the contraction measured by tdm_prepare on 64
                              seeded right-hand sides (four corrections: the size of the second
                              per unit of the first).  Each tile then makes its first correction,
                              writes X and is checked during the next tile's first exchange; a
                              tile that fails is solved again with the tests after every
                              correction.  Plans too large to calibrate cheaply
                              (n > ~350000 uses fewer columns, n > ~2.8e6 none) keep contraction 1.
                              tdm_info reports both. */
  int flags;         /* reserved, must be 0 */
  int tile_rhs;      /* TDM_FP32_REFINED: right-hand sides per tile of the solve kernel, 4, 8 or
                        16; 0 (automatic) = 8 where the shape fits (the shape rule falls back to
                        other widths when a requested one does not fit the system size) */
} tdm_options;

typedef struct {
  int64_t n;               /* system size */
  int32_t block_rows;      /* rows per block */
  int32_t num_blocks;      /* M = ceil(n / block_rows); separators = M - 1 */
  int32_t dominant;        /* 1 if |b_i| >= |a_{i-1}| + |a_i| for all i with one strict
                              inequality (Theorem 4: the method is then stable) */
  int32_t refine_steps;    /* corrections of a TDM_FP32_REFINED solve: 1..4, or -1 (tested per tile) */
  double max_abs_z;        /* max |Z^R|, |Z^L| ratio between neighbouring separators */
  double min_abs_pivot;    /* smallest |pivot| met in prepare, relative to ||A||_inf */
  int32_t device_error;    /* device-side error code of the last solves (0 = none,
                              1 = a TMA transfer timed out, 2 = refinement cap reached
                              before the convergence test passed, 3 = a CTA of a
                              cooperative refined launch waited too long for its group) */
  int32_t tile_rhs;        /* the plan's tile_rhs option (0 = automatic) */
  int32_t general;         /* 1 for a plan of tdm_prepare_general (a nonsymmetric matrix) */
  float contraction;       /* TDM_FP32_REFINED per-tile test: estimated relative error left by
                              the first correction per unit of its size (1 = not calibrated) */
} tdm_info;

/* tdm_prepare -- Algorithm 3/4, step 1 (Sections 3.3-3.4; eqs. green_v, z_vector).
 *   a      device, n-1 binary64 off-diagonal entries (may be NULL when n == 1)
 *   b      device, n binary64 diagonal entries
 *   n      system size, 1 <= n <= 2^26
 *   opt    may be NULL (all automatic)
 *   stream enqueue the preparation on this stream; the call waits for it
 *   out    receives the handle; the plan owns its device memory until
 *          tdm_destroy.  a and b may be freed after the call returns.
 * Errors: TDM_ERR_INVALID_ARG (n out of range, null pointers, 8-byte
 * misalignment), TDM_ERR_SINGULAR (nondegeneracy violated, Section 2),
 * TDM_ERR_NO_MEMORY, TDM_ERR_CUDA.  On error *out is set to NULL.
 * With refine_steps = 0 the call also runs one calibration solve (see tdm_options). */
tdm_status tdm_prepare(const double* a, const double* b, int64_t n,
                       const tdm_options* opt, void* stream, tdm_handle* out);

/* tdm_prepare_general -- a nonsymmetric tridiagonal A, symmetrized by the
 * diagonal similarity of Section 3.5: with T = diag(t), t_{k+1} = t_k
 * (sub_k / sup_k)^(1/2), T^-1 A T is symmetric, and the plan of that matrix
 * is prepared with every factor of T folded into its coefficients, so that
 * the solves return x = A^-1 F.
 *   sub    device, n-1 binary64 entries A[k+1][k]
 *   diag   device, n binary64 entries A[k][k]
 *   sup    device, n-1 binary64 entries A[k][k+1]
 *   n, opt, stream, out as for tdm_prepare (tile_rhs and refine_steps are unused).
 * Requires sub_k * sup_k > 0 for every k (the similarity exists); the factors
 * of T within one block must stay finite in binary32 for TDM_FP32 solves.
 * Errors: TDM_ERR_INVALID_ARG also when some sub_k * sup_k <= 0; the others as
 * for tdm_prepare.  A general plan serves TDM_FP64 and TDM_FP32 solves,
 * batched or not; TDM_FP32_REFINED solves and tdm_solve_backward return
 * TDM_ERR_NOT_IMPLEMENTED for it. */
tdm_status tdm_prepare_general(const double* sub, const double* diag, const double* sup, int64_t n,
                               const tdm_options* opt, void* stream, tdm_handle* out);

/* tdm_solve -- Algorithm 3/4, step 2 for every column (Theorem 2, Lemma 1).
 *   F   device, [n][ldF], dtype per `prec` (binary64 for TDM_FP64, else binary32)
 *   X   device, [n][ldX], binary64 for TDM_FP64 and TDM_FP32_REFINED, binary32
 *       for TDM_FP32.  F and X must not overlap.
 *   N   number of right-hand sides; N == 0 is a no-op.
 * Pointers must be 16-byte aligned and ldF, ldX >= N.
 * Sizes: one thread-block cluster holds all n rows of a tile of right-hand
 * sides up to n = 1024 * block_rows (TDM_FP32_REFINED: 65536).  A larger
 * symmetric plan is solved in two levels (Lemma 1 one level up): segments of
 * at most 1024 * block_rows rows, each by a plan of its own, and the values at
 * the rows between them from a reduced tridiagonal plan; X then takes one more
 * read and write.  tdm_solve_batched solves such plans by their two-level
 * solve, one after the other on the stream, beside the batched layout of the
 * others; tdm_solve_batched_noalloc (whose two-level solve would allocate)
 * and general plans beyond the limit return TDM_ERR_NOT_IMPLEMENTED.
 * Errors: TDM_ERR_INVALID_ARG, TDM_ERR_NOT_IMPLEMENTED, TDM_ERR_CUDA. */
tdm_status tdm_solve(tdm_handle h, const void* F, int64_t ldF, void* X, int64_t ldX,
                     int64_t N, tdm_precision prec, void* stream);

/* tdm_solve_host -- tdm_solve for right-hand sides and solutions in HOST
 * memory (no counterpart in the paper: the copies of a series that does not
 * live on the device).  The columns are cut into chunks of `chunk` columns
 * (0: about N/4, at least 2048; rounded up to a multiple of 16); each chunk is
 * copied in, solved and copied out on separate streams, with two device
 * staging buffers per direction that the plan keeps (sized for the largest
 * chunk used), so that the copies overlap the solves.
 *   F   host, [n][ldF], dtype per `prec`; X host, [n][ldX], dtype per `prec`.
 *       Pinned memory lets the copies run asynchronously and overlap; pageable
 *       memory works, with copies that the driver stages.
 *   stream  all work starts after the work already enqueued on it, and the
 *       stream completes when the last column of X has reached the host: the
 *       caller synchronizes the stream before reading X.
 * Calls on one plan must be ordered (one stream, or synchronized): they share
 * the staging buffers.  Not capturable in a CUDA graph.
 * Errors: TDM_ERR_INVALID_ARG (null or overlapping F and X, ld < N, chunk < 0),
 * TDM_ERR_NOT_IMPLEMENTED (refined solve of a general plan; stream capture),
 * TDM_ERR_NO_MEMORY, TDM_ERR_CUDA. */
tdm_status tdm_solve_host(tdm_handle h, const void* F, int64_t ldF, void* X, int64_t ldX, int64_t N,
                          int64_t chunk, tdm_precision prec, void* stream);

/* tdm_solve_batched -- many distinct constant matrices, each with its own
 * block of right-hand sides (the per-mode series of the Fourier method,
 * Section 4, eqs. series_fft, poisson_end), by the refined persistent kernel
 * in the layout tdm_set_batched_strategy selects.
 *   hs[k], F[k], ldF[k], X[k], ldX[k], N[k] for k = 0..count-1, with the same
 *   meaning as for tdm_solve (host arrays of device pointers).  All plans must
 *   have the same block_rows.  Work lists are built and uploaded on the first
 *   call with an argument set and kept until one of its plans is destroyed;
 *   later calls (and CUDA-graph replays of a captured call) upload nothing.
 * Errors: as tdm_solve, plus TDM_ERR_INVALID_ARG for mixed block_rows. */
tdm_status tdm_solve_batched(const tdm_handle* hs, int count,
                             const void* const* F, const int64_t* ldF,
                             void* const* X, const int64_t* ldX, const int64_t* N,
                             tdm_precision prec, void* stream);

/* tdm_set_batched_strategy -- how tdm_solve_batched lays out refined work,
 * process-wide, from the next call on:
 *   3  (default) by rule: 0 when the batch needs at most four launch classes
 *      (kernel shape and cluster width), else 2;
 *   2  one single-series launch per series, biggest first, round robin over
 *      the caller's stream and three helper streams that fork from it and
 *      join it again;
 *   0  one persistent launch per kernel shape and cluster width over a work
 *      list of tiles (a cluster takes one tile of one series at a time),
 *      spread over the same streams;
 *   1  one persistent launch per kernel shape and correction schedule: the
 *      clusters are as wide as the widest series needs, and each walks a list
 *      of units in which tiles of several series run side by side, each on an
 *      aligned power-of-two group of CTAs.
 *   4  one cooperative persistent launch per kernel shape over every CTA the
 *      GPU holds at once, without clusters: each series keeps its own
 *      partition (g CTAs), its tiles are cut into runs placed on windows of g
 *      consecutive CTAs, and each run's CTAs exchange values through global
 *      memory and a barrier counter of the run.
 * Under each, a series with a fixed or calibrated refinement gets the result
 * of its own tdm_solve, bit for bit (under 4 any series does); under 1, a plan with the uncalibrated
 * per-tile test (refine_steps = -1 requested), and a unit whose speculative
 * check fails, run four corrections and a convergence check.
 * Errors: TDM_ERR_INVALID_ARG for any other value. */
tdm_status tdm_set_batched_strategy(int strategy);

/* tdm_solve_batched_noalloc -- tdm_solve_batched with TDM_FP32_REFINED for
 * callers that must not allocate: the call allocates no device or host memory
 * (no cudaMalloc, cudaMallocHost, cudaFree).  The paper has no counterpart:
 * this is a memory-management variant of the batched solve, not a step of the
 * method.  Callers who cannot allocate: one whose device memory is held by
 * its own pool (a cudaMalloc could fail although the pool has room); one in a
 * loop overlapping several streams (allocation and release may synchronize the
 * device); one passing new F / X pointers every call (tdm_solve_batched keeps
 * one work list per argument set until a plan is destroyed).
 *   Arguments as tdm_solve_batched: hs[k], F[k] (binary32), ldF[k], X[k]
 *   (binary64), ldX[k], N[k]; all plans on one device, same block_rows.
 * The work list -- one item per tile of right-hand sides, ceil(N[k] / R)
 * items for series k, R = 4, 8 or 16 by the series' size -- is written into a
 * fixed device array of TDM_NOALLOC_MAX_TILES items (384 KiB), one per device,
 * shared by all calls on that device and keeping the last call's items.
 *   - The first call on a device sets it up (looks up the array's device
 *     address, loading the library's device code there); make it before any
 *     stream capture.
 *   - Calls that overlap on the device (different streams with no ordering
 *     between them) race on the array: serialize them on one stream, or
 *     order the streams with events.
 *   - The items are copied from a static host array in pageable memory; the
 *     driver may make that copy wait for the stream's earlier work, so the
 *     call can block the host until then.
 * Not capturable: under stream capture the call returns
 * TDM_ERR_NOT_IMPLEMENTED and enqueues nothing (a captured copy would read the
 * host array again at every replay, after later calls have refilled it).
 * Errors: as tdm_solve_batched; TDM_ERR_TOO_LARGE when the items of one call
 * exceed TDM_NOALLOC_MAX_TILES (nothing is enqueued); TDM_ERR_NOT_IMPLEMENTED
 * under stream capture. */
#define TDM_NOALLOC_MAX_TILES 4096
tdm_status tdm_solve_batched_noalloc(const tdm_handle* hs, int count,
                                     const float* const* F, const int64_t* ldF,
                                     double* const* X, const int64_t* ldX, const int64_t* N,
                                     void* stream);

/* tdm_solve_backward -- gradients of a scalar loss L through X = A^{-1} F.
 * A is symmetric, so the adjoint system A^T Lambda = W is another solve with
 * the same plan (Lemma 2).  With W = dL/dX and X the forward solution:
 *   dF = Lambda,  db_i = -sum_r Lambda_ir X_ir,
 *   da_i = -sum_r (Lambda_ir X_{i+1,r} + Lambda_{i+1,r} X_ir).
 *   W      device [n][ld]: binary64 (TDM_FP64), binary32 (TDM_FP32, TDM_FP32_REFINED)
 *   X      device [n][ld]: the forward solution, binary64 (TDM_FP64, TDM_FP32_REFINED)
 *          or binary32 (TDM_FP32)
 *   dF     device [n][ld], the dtype of X; receives Lambda (for TDM_FP32_REFINED the
 *          refined solve of W: binary64 accuracy at binary32 input)
 *   da, db device binary64 arrays of n-1 and n entries, or NULL to skip
 * The row sums over right-hand sides are accumulated in binary64 in a fixed
 * order (deterministic).
 * Errors: TDM_ERR_INVALID_ARG, TDM_ERR_NOT_IMPLEMENTED (general plans), TDM_ERR_CUDA. */
tdm_status tdm_solve_backward(tdm_handle h, const void* W, const void* X, int64_t ld,
                              int64_t N, void* dF, double* da, double* db,
                              tdm_precision prec, void* stream);

/* tdm_algorithm2 -- Algorithm 2 (Section 3.1): selected components of every
 * solution as dense products, X[k][r] = sum_i G_k(i) F[i][r] for P components
 * k, with G_k = A^{-1} e_k the inverse rows (eq. green_v, Lemma 2; a caller
 * obtains them from tdm_solve on unit right-hand sides).  The product runs on
 * the tensor cores (tcgen05.mma, TF32 inputs, binary32 accumulation in tensor
 * memory) as three TF32 products of the operands' TF32 heads and binary32
 * tails; each binary32 accumulation covers at most 1024 rows of K, and the
 * partial sums are added in binary32 pairs.
 *   G     device, [n][ldG] binary64: column k is G_k (ldG >= P)
 *   F     device, [n][ldF] binary32 right-hand sides; 16-byte aligned, ldF a
 *         multiple of 4
 *   X     device, [P][ldX] binary32, receives the components (ldX >= N)
 *   work  device workspace of at least tdm_algorithm2_workspace(min(P, 512), n, N)
 *         bytes, 256-byte aligned; calls that share it must be ordered
 * Components are processed 512 at a time.  Asynchronous on `stream`; a bounded
 * device wait that gave up is reported by tdm_algorithm2_status.
 * Errors: TDM_ERR_INVALID_ARG (sizes, strides, alignment, workspace too small),
 * TDM_ERR_NOT_IMPLEMENTED (F cannot be described to the copy engine),
 * TDM_ERR_CUDA. */
size_t tdm_algorithm2_workspace(int64_t P, int64_t n, int64_t N);
tdm_status tdm_algorithm2(const double* G, int64_t ldG, int64_t P, int64_t n, const float* F, int64_t ldF,
                          int64_t N, float* X, int64_t ldX, void* work, size_t work_bytes, void* stream);
/* tdm_algorithm2_status -- the device error word of the last tdm_algorithm2 call
 * with this workspace and sizes (0 = none, 1 = a bounded wait gave up);
 * synchronizes the stream. */
tdm_status tdm_algorithm2_status(const void* work, int64_t P, int64_t n, int64_t N, void* stream,
                                 int* device_error);

/* tdm_adi_rhs -- the right-hand side of one Peaceman-Rachford half step
 * (Section 4b, eqs. adi_iter, adi_iter2), scaled by h^2, in one pass:
 *   R[a][b*S + s] = c v[a][b][s] + h2 f[a][b][s] + v[a][b-1][s] + v[a][b+1][s]
 * (v = 0 beyond b's ends), the series of tdm_solve along a whose columns are
 * the lines b of the problems s (c = omega h^2 - 2, h2 = h^2).
 *   v, f   device; element (a, b, s) at a*va + b*vb + s (resp. fa, fb), unit
 *          stride along s, so transposed views of [a][b][s] arrays are
 *          accepted; binary64 when in_f64, else binary32.
 *   R      device, [na][ldR], ldR >= nb*S; binary64 when out_f64, else binary32
 *          (binary32 in with binary64 out is not offered).  Must not overlap
 *          v or f.
 * Arithmetic: binary64 results are summed in binary64; binary64 inputs with
 * binary32 results are summed in pairs of binary32 numbers (about 2^-47 of
 * the terms, then one rounding); binary64 arithmetic instead for a run of
 * four lines b of one (a, s) whose inputs include a value outside the pairs'
 * range (0 < |x| < 2^-74, |x| >= 2^128, non-finite), and everywhere when c or
 * h2 is nonzero and outside [2^-60, 2^60]; binary32 inputs are summed in
 * binary32.  Asynchronous on `stream`.
 * Errors: TDM_ERR_INVALID_ARG (negative sizes, null pointers, ldR < nb*S,
 * nb*S above 2^31 - 1, the binary32-to-binary64 combination), TDM_ERR_CUDA.
 * Empty sizes return TDM_OK without a launch. */
tdm_status tdm_adi_rhs(const void* v, int64_t va, int64_t vb, const void* f, int64_t fa, int64_t fb, int64_t na,
                       int64_t nb, int64_t S, double c, double h2, int in_f64, void* R, int64_t ldR, int out_f64,
                       void* stream);

/* tdm_selftest_wait_timeout -- a check of the failure path of the solve
 * kernels' bounded waits (no counterpart in the paper): one CTA waits on an
 * mbarrier that nothing arrives at, gives up after `limit_cycles` clock
 * cycles (1 .. 2^31), records the timeout in a device word and exits; the
 * context stays usable.  Returns TDM_ERR_TIMEOUT when the wait gave up as it
 * must, TDM_OK if it did not, TDM_ERR_INVALID_ARG for a limit out of range.
 * Synchronizes the stream. */
tdm_status tdm_selftest_wait_timeout(int64_t limit_cycles, void* stream);

/* tdm_selftest_group_timeout -- the same check for the group barrier of the
 * cooperative launches (no counterpart in the paper): in a cooperative grid
 * of two CTAs forming one group, CTA 1 never arrives; CTA 0 arrives, polls the
 * group's counter `limit_polls` times (1 .. 2^24), gives up, records device
 * error 3 and exits; the context stays usable.  Returns TDM_ERR_TIMEOUT when
 * the wait gave up as it must, TDM_OK if it did not, TDM_ERR_INVALID_ARG for a
 * limit out of range.  Synchronizes the stream. */
tdm_status tdm_selftest_group_timeout(int64_t limit_polls, void* stream);

/* tdm_get_info -- plan properties and the device status of the last solve
 * (synchronizes with it). */
tdm_status tdm_get_info(tdm_handle h, tdm_info* info);

/* tdm_destroy -- releases the plan's device memory (synchronizes first).
 * NULL is accepted and ignored. */
tdm_status tdm_destroy(tdm_handle h);

/* tdm_status_string -- static, human-readable name of a status code. */
const char* tdm_status_string(tdm_status s);

#ifdef __cplusplus
}
#endif

#endif /* TDM_H */
