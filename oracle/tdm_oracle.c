/*
 * tdm_oracle.c -- plain, slow CPU oracle for the series A X_n = F_n, n = 1..N,
 * with one symmetric tridiagonal A (diagonal b_i, off-diagonal a_i), as stated
 * in Section 2 (eq. main_eq3) of Terekhov, "Parallel dichotomy algorithm for
 * solving tridiagonal SLAEs".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * The dichotomy method reaches X = A^{-1} F exactly in exact arithmetic
 * (Lemma 1 and Theorem 2 are identities), so this oracle is that plain
 * definition computed without any of the method's machinery:
 *
 *   oracle_thomas_f64   the textbook sweep (LU of the tridiagonal matrix,
 *                       forward elimination, back substitution) in binary64,
 *                       the sequential method the paper compares against
 *                       (Section 3.3, T_1 = 8n; Theorem 4 cites the sweep).
 *   oracle_solve_hi     oracle_thomas_f64 followed by iterative refinement in
 *                       which the residual F - A x is formed and the iterate
 *                       accumulated in long double.  This is the reference
 *                       for every floating-point tolerance.
 *   oracle_gauss_ld     dense Gaussian elimination with partial pivoting in
 *                       long double: an independent check for small n.
 *   oracle_matvec_ld    y = A x in long double (residuals, backward errors).
 *   oracle_grad_ld      gradients of L = sum(W * X), X = A^{-1} F, from the
 *                       adjoint solve; A = A^T (Lemma 2), so the adjoint
 *                       system is another solve with the same A.
 *
 * Layout: F, X, W are row-major [n][ld] with the right-hand sides contiguous,
 * element (row i, rhs r) at F[i*ld + r]; a has n-1 entries, b has n.
 * Every function returns 0 on success, -1 on an invalid argument and -2 when a
 * pivot is exactly zero.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ldbl;

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Textbook sweep.  Pivots d_i = b_i - a_{i-1}^2 / d_{i-1} do not depend on the
 * right-hand side, so they are formed once; every column then gets
 *   g_0 = f_0,            g_i = f_i - (a_{i-1}/d_{i-1}) g_{i-1},
 *   x_{n-1} = g_{n-1}/d_{n-1},   x_i = (g_i - a_i x_{i+1}) / d_i.
 * The columns are independent; OpenMP splits them over threads. */
int oracle_thomas_f64(int64_t n, const double* a, const double* b,
                      const double* F, int64_t ldF, int64_t N,
                      double* X, int64_t ldX, int nthreads) {
  if (n < 1 || N < 0 || ldF < N || ldX < N || !b || (n > 1 && !a)) return -1;
  if (N == 0) return 0;
  if (!F || !X) return -1;
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* l = (double*)malloc(sizeof(double) * (size_t)n);
  if (!d || !l) { free(d); free(l); return -1; }
  int bad = 0;
  d[0] = b[0];
  l[0] = 0.0;
  if (d[0] == 0.0) bad = 1;
  for (int64_t i = 1; i < n && !bad; i++) {
    l[i] = a[i - 1] / d[i - 1];
    d[i] = b[i] - l[i] * a[i - 1];
    if (d[i] == 0.0) bad = 1;
  }
  if (bad) { free(d); free(l); return -2; }
  if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
  for (int64_t r = 0; r < N; r++) {
    /* forward elimination, written in place into X */
    X[r] = F[r];
    for (int64_t i = 1; i < n; i++)
      X[i * ldX + r] = F[i * ldF + r] - l[i] * X[(i - 1) * ldX + r];
    /* back substitution */
    X[(n - 1) * ldX + r] = X[(n - 1) * ldX + r] / d[n - 1];
    for (int64_t i = n - 2; i >= 0; i--)
      X[i * ldX + r] = (X[i * ldX + r] - a[i] * X[(i + 1) * ldX + r]) / d[i];
  }
  free(d);
  free(l);
  return 0;
}

/* y = A x in long double.  x, y are [n][ld] in long double. */
static void matvec_ld(int64_t n, const double* a, const double* b,
                      const ldbl* x, int64_t ldx, int64_t N, ldbl* y, int64_t ldy) {
  for (int64_t i = 0; i < n; i++) {
    for (int64_t r = 0; r < N; r++) {
      ldbl s = (ldbl)b[i] * x[i * ldx + r];
      if (i > 0) s += (ldbl)a[i - 1] * x[(i - 1) * ldx + r];
      if (i + 1 < n) s += (ldbl)a[i] * x[(i + 1) * ldx + r];
      y[i * ldy + r] = s;
    }
  }
}

/* y = A x in long double, with x and y given in binary64 (y is rounded once). */
int oracle_matvec_ld(int64_t n, const double* a, const double* b,
                     const double* x, int64_t ldx, int64_t N, double* y, int64_t ldy) {
  if (n < 1 || N < 0 || ldx < N || ldy < N || !b || (n > 1 && !a)) return -1;
  for (int64_t i = 0; i < n; i++) {
    for (int64_t r = 0; r < N; r++) {
      ldbl s = (ldbl)b[i] * (ldbl)x[i * ldx + r];
      if (i > 0) s += (ldbl)a[i - 1] * (ldbl)x[(i - 1) * ldx + r];
      if (i + 1 < n) s += (ldbl)a[i] * (ldbl)x[(i + 1) * ldx + r];
      y[i * ldy + r] = (double)s;
    }
  }
  return 0;
}

/* x_0 = sweep(F);  for k = 1..steps:  r = F - A x_k (long double),
 * x_{k+1} = x_k + sweep(r rounded to binary64)  (x kept in long double).
 * The result is rounded once to binary64.  Columns are processed in groups
 * so that the long double work arrays stay small. */
int oracle_solve_hi(int64_t n, const double* a, const double* b,
                    const double* F, int64_t ldF, int64_t N,
                    double* X, int64_t ldX, int steps, int nthreads) {
  if (n < 1 || N < 0 || ldF < N || ldX < N || steps < 0 || !b || (n > 1 && !a)) return -1;
  if (N == 0) return 0;
  if (!F || !X) return -1;
  const int64_t G = 64; /* columns per group */
  int status = 0;
  if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic)
#endif
  for (int64_t c0 = 0; c0 < N; c0 += G) {
    int64_t g = (N - c0 < G) ? (N - c0) : G;
    ldbl* x = (ldbl*)malloc(sizeof(ldbl) * (size_t)(n * g));
    ldbl* ax = (ldbl*)malloc(sizeof(ldbl) * (size_t)(n * g));
    double* r = (double*)malloc(sizeof(double) * (size_t)(n * g));
    double* d = (double*)malloc(sizeof(double) * (size_t)(n * g));
    int st = (x && ax && r && d) ? 0 : -1;
    if (!st) {
      for (int64_t i = 0; i < n; i++)
        for (int64_t c = 0; c < g; c++) r[i * g + c] = F[i * ldF + c0 + c];
      st = oracle_thomas_f64(n, a, b, r, g, g, d, g, 1);
    }
    if (!st) {
      for (int64_t i = 0; i < n * g; i++) x[i] = (ldbl)d[i];
      for (int k = 0; k < steps && !st; k++) {
        matvec_ld(n, a, b, x, g, g, ax, g);
        for (int64_t i = 0; i < n; i++)
          for (int64_t c = 0; c < g; c++)
            r[i * g + c] = (double)((ldbl)F[i * ldF + c0 + c] - ax[i * g + c]);
        st = oracle_thomas_f64(n, a, b, r, g, g, d, g, 1);
        if (!st)
          for (int64_t i = 0; i < n * g; i++) x[i] += (ldbl)d[i];
      }
    }
    if (!st)
      for (int64_t i = 0; i < n; i++)
        for (int64_t c = 0; c < g; c++) X[i * ldX + c0 + c] = (double)x[i * g + c];
    free(x); free(ax); free(r); free(d);
    if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
      status = st;
    }
  }
  return status;
}

/* Dense Gaussian elimination with partial pivoting in long double.
 * Adense is n x n row-major (binary64 input, promoted); F, X are [n][ld]. */
int oracle_gauss_ld(int64_t n, const double* Adense, const double* F, int64_t ldF,
                    int64_t N, double* X, int64_t ldX) {
  if (n < 1 || N < 0 || ldF < N || ldX < N || !Adense) return -1;
  ldbl* A = (ldbl*)malloc(sizeof(ldbl) * (size_t)(n * n));
  ldbl* B = (ldbl*)malloc(sizeof(ldbl) * (size_t)(n * (N > 0 ? N : 1)));
  if (!A || !B) { free(A); free(B); return -1; }
  for (int64_t i = 0; i < n * n; i++) A[i] = (ldbl)Adense[i];
  for (int64_t i = 0; i < n; i++)
    for (int64_t r = 0; r < N; r++) B[i * N + r] = (ldbl)F[i * ldF + r];
  int st = 0;
  for (int64_t k = 0; k < n && !st; k++) {
    int64_t p = k;
    ldbl best = fabsl(A[k * n + k]);
    for (int64_t i = k + 1; i < n; i++)
      if (fabsl(A[i * n + k]) > best) { best = fabsl(A[i * n + k]); p = i; }
    if (best == 0.0L) { st = -2; break; }
    if (p != k) {
      for (int64_t j = 0; j < n; j++) { ldbl t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
      for (int64_t r = 0; r < N; r++) { ldbl t = B[k * N + r]; B[k * N + r] = B[p * N + r]; B[p * N + r] = t; }
    }
    for (int64_t i = k + 1; i < n; i++) {
      ldbl m = A[i * n + k] / A[k * n + k];
      if (m == 0.0L) continue;
      for (int64_t j = k; j < n; j++) A[i * n + j] -= m * A[k * n + j];
      for (int64_t r = 0; r < N; r++) B[i * N + r] -= m * B[k * N + r];
    }
  }
  if (!st) {
    for (int64_t r = 0; r < N; r++) {
      for (int64_t i = n - 1; i >= 0; i--) {
        ldbl s = B[i * N + r];
        for (int64_t j = i + 1; j < n; j++) s -= A[i * n + j] * B[j * N + r];
        B[i * N + r] = s / A[i * n + i];
      }
    }
    for (int64_t i = 0; i < n; i++)
      for (int64_t r = 0; r < N; r++) X[i * ldX + r] = (double)B[i * N + r];
  }
  free(A);
  free(B);
  return st;
}

/* Gradients of L = sum_{i,r} W_ir X_ir with A X = F (A symmetric):
 *   Lambda = A^{-T} W = A^{-1} W          (adjoint solve, same matrix),
 *   dL/dF  = Lambda,
 *   dL/db_i = -sum_r Lambda_ir X_ir,
 *   dL/da_i = -sum_r (Lambda_ir X_{i+1,r} + Lambda_{i+1,r} X_ir).
 * X and Lambda come from oracle_solve_hi; the sums are accumulated in long
 * double.  dF, da, db may each be NULL. */
int oracle_grad_ld(int64_t n, const double* a, const double* b,
                   const double* F, const double* W, int64_t ld, int64_t N,
                   double* dF, double* da, double* db, int steps, int nthreads) {
  if (n < 1 || N < 0 || ld < N || !b || (n > 1 && !a)) return -1;
  double* X = (double*)malloc(sizeof(double) * (size_t)(n * (N > 0 ? N : 1)));
  double* L = (double*)malloc(sizeof(double) * (size_t)(n * (N > 0 ? N : 1)));
  if (!X || !L) { free(X); free(L); return -1; }
  int st = 0;
  if (N > 0) {
    st = oracle_solve_hi(n, a, b, F, ld, N, X, N, steps, nthreads);
    if (!st) st = oracle_solve_hi(n, a, b, W, ld, N, L, N, steps, nthreads);
  }
  if (!st) {
    if (dF)
      for (int64_t i = 0; i < n; i++)
        for (int64_t r = 0; r < N; r++) dF[i * ld + r] = L[i * N + r];
    if (db)
      for (int64_t i = 0; i < n; i++) {
        ldbl s = 0.0L;
        for (int64_t r = 0; r < N; r++) s += (ldbl)L[i * N + r] * (ldbl)X[i * N + r];
        db[i] = (double)(-s);
      }
    if (da)
      for (int64_t i = 0; i + 1 < n; i++) {
        ldbl s = 0.0L;
        for (int64_t r = 0; r < N; r++)
          s += (ldbl)L[i * N + r] * (ldbl)X[(i + 1) * N + r] + (ldbl)L[(i + 1) * N + r] * (ldbl)X[i * N + r];
        da[i] = (double)(-s);
      }
  }
  free(X);
  free(L);
  return st;
}
