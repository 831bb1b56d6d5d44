"""CPU oracle for the series A X_n = F_n with one symmetric tridiagonal A.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this package; the product path never imports
it.  It shares no code with the CUDA library.

Contents
--------
C part (``tdm_oracle.c``, built on demand with gcc):
  thomas_f64   textbook sweep in binary64 (Section 3.3: sequential sweep, T_1 = 8n)
  solve_hi     sweep + iterative refinement with long double residuals
  gauss_ld     dense partial-pivoting elimination in long double
  matvec_ld    A x in long double
  grad_ld      dL/dF, dL/da, dL/db of L = sum(W * X) via the adjoint solve (Lemma 2)
numpy part (this file):
  dense                 the matrix of Section 2 (eq. main_eq3)
  eigen_closed_form     eigen right-hand sides of -u'' + s u with their exact
                        solutions (Section 4, eq. SLAU_FFT; sine eigenvectors)
  omega_levels          the level sets Omega_i of eq. omega_i (Section 3.4)
  dichotomy_ld          Algorithm 3 + Algorithm 1 in long double, step by step
                        (Theorem 2, eqs. theor_2, beta_symn, z_vector, matrixbrl)
  z_vectors             Z^R_k, Z^L_k from eq. z_vector (for the Theorem 4 bound)
  explicit_inverse      the explicit inverse of Section 3.6 (eqs. x1-x3),
                        symmetric case
  algorithm2            selected solution components as G_k^T F (Algorithm 2, Section 3.1)
  thomas_general        the sweep for a general (nonsymmetric) tridiagonal matrix
  symmetrizer           the diagonal similarity that symmetrizes it (Section 3.5)
Parity is pinned for every function here by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_tdm.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle_tdm.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int
            lib.oracle_thomas_f64.argtypes = [i64, dp, dp, dp, i64, i64, dp, i64, ip]
            lib.oracle_solve_hi.argtypes = [i64, dp, dp, dp, i64, i64, dp, i64, ip, ip]
            lib.oracle_gauss_ld.argtypes = [i64, dp, dp, i64, i64, dp, i64]
            lib.oracle_matvec_ld.argtypes = [i64, dp, dp, dp, i64, i64, dp, i64]
            lib.oracle_grad_ld.argtypes = [i64, dp, dp, dp, dp, i64, i64, dp, dp, dp, ip, ip]
            lib.oracle_max_threads.argtypes = []
            for f in ("oracle_thomas_f64", "oracle_solve_hi", "oracle_gauss_ld",
                      "oracle_matvec_ld", "oracle_grad_ld", "oracle_max_threads"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(x):
    return None if x is None else x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _check(status, what):
    if status == -2:
        raise ZeroDivisionError(f"{what}: zero pivot (singular matrix)")
    if status != 0:
        raise ValueError(f"{what}: invalid argument (status {status})")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _as2d(F):
    F = _f64(F)
    return (F[:, None], True) if F.ndim == 1 else (F, False)


def thomas_f64(a, b, F, threads: int | None = None):
    """Textbook sweep in binary64 for every column of F (shape (n,) or (n, N))."""
    a, b = _f64(a), _f64(b)
    F, squeeze = _as2d(F)
    n, N = F.shape
    X = np.empty_like(F)
    t = threads or max_threads()
    _check(_load().oracle_thomas_f64(n, _p(a), _p(b), _p(F), N, N, _p(X), N, t), "thomas_f64")
    return X[:, 0] if squeeze else X


def solve_hi(a, b, F, steps: int = 3, threads: int | None = None):
    """Sweep plus `steps` refinement steps with long double residuals."""
    a, b = _f64(a), _f64(b)
    F, squeeze = _as2d(F)
    n, N = F.shape
    X = np.empty_like(F)
    t = threads or max_threads()
    _check(_load().oracle_solve_hi(n, _p(a), _p(b), _p(F), N, N, _p(X), N, steps, t), "solve_hi")
    return X[:, 0] if squeeze else X


def dense(a, b):
    """The n x n matrix of Section 2: diagonal b, both off-diagonals a."""
    a, b = _f64(a), _f64(b)
    n = b.shape[0]
    A = np.diag(b)
    if n > 1:
        A[np.arange(n - 1), np.arange(1, n)] = a
        A[np.arange(1, n), np.arange(n - 1)] = a
    return A


def gauss_ld(Adense, F):
    """Dense partial-pivoting elimination in long double (any square matrix)."""
    A = _f64(Adense)
    F, squeeze = _as2d(F)
    n, N = F.shape
    X = np.empty_like(F)
    _check(_load().oracle_gauss_ld(n, _p(A), _p(F), N, N, _p(X), N), "gauss_ld")
    return X[:, 0] if squeeze else X


def matvec_ld(a, b, X):
    """A X formed in long double, rounded once to binary64."""
    a, b = _f64(a), _f64(b)
    X, squeeze = _as2d(X)
    n, N = X.shape
    Y = np.empty_like(X)
    _check(_load().oracle_matvec_ld(n, _p(a), _p(b), _p(X), N, N, _p(Y), N), "matvec_ld")
    return Y[:, 0] if squeeze else Y


def grad_ld(a, b, F, W, steps: int = 3, threads: int | None = None):
    """(dL/dF, dL/da, dL/db) for L = sum(W * X), X = A^{-1} F."""
    a, b = _f64(a), _f64(b)
    F, W = _f64(F), _f64(W)
    n, N = F.shape
    dF = np.empty_like(F)
    da = np.empty(max(n - 1, 1))
    db = np.empty(n)
    t = threads or max_threads()
    _check(_load().oracle_grad_ld(n, _p(a), _p(b), _p(F), _p(W), N, N, _p(dF), _p(da), _p(db), steps, t),
           "grad_ld")
    return dF, da[: n - 1], db


# ----------------------------------------------------------------------------
# Closed forms (Section 4)
# ----------------------------------------------------------------------------

def eigen_closed_form(n: int, b_value: float, ks):
    """Eigen right-hand sides for a_i = -1, b_i = b_value (= 2 + s).

    Section 4 (eq. SLAU_FFT) separates variables with sine modes: the vector
    v_k(i) = sin(pi k i / (n+1)), i = 1..n, is an eigenvector of
    tridiag(-1, 2, -1) with eigenvalue 4 sin^2(pi k / (2(n+1))).  Hence for
    A = tridiag(-1, 2 + s, -1) the right-hand side F = v_k has the solution
    X = v_k / lambda_k, lambda_k = s + 4 sin^2(pi k / (2(n+1))).

    s is taken as (b_value - 2), exact in binary64 (Sterbenz), and the sine
    arguments are reduced exactly in integers, ((k i) mod 2(n+1)).  Returns
    (F, X, lam) with F, X of shape (n, len(ks)) in binary64; X is evaluated
    in long double and rounded once.
    """
    ks = np.asarray(ks, dtype=np.int64)
    i = np.arange(1, n + 1, dtype=np.int64)
    m = (np.outer(i, ks) % (2 * (n + 1))).astype(np.longdouble)
    pi = np.longdouble(np.pi) + np.longdouble(1.2246467991473532e-16)  # pi to ~long double
    v = np.sin(pi * m / np.longdouble(n + 1))
    s = np.longdouble(np.float64(b_value) - 2.0)
    lam = s + 4 * np.sin(pi * ks.astype(np.longdouble) / np.longdouble(2 * (n + 1))) ** 2
    F = v.astype(np.float64)
    X = (F.astype(np.longdouble) / lam).astype(np.float64)
    return F, X, lam.astype(np.float64)


# ----------------------------------------------------------------------------
# Level sets of the dichotomy algorithm (Section 3.4, eq. omega_i)
# ----------------------------------------------------------------------------

def omega_levels(p: int):
    """Omega_i, i = 1..floor(log2 p) + 1, as lists of separator numbers 1..p.

    Omega_i collects the separators j = 2^(floor(log2 p) + 1 - i) * k,
    k = 1..2^i - 1 (those within 1..p), minus the ones already in an earlier
    level.  Every separator 1..p lands in exactly one level.
    """
    if p < 1:
        return []
    top = int(np.floor(np.log2(p))) + 1
    seen, levels = set(), []
    for i in range(1, top + 1):
        step = 2 ** (top - i)
        lev = [step * k for k in range(1, 2 ** i) if step * k <= p and step * k not in seen]
        seen.update(lev)
        levels.append(lev)
    return levels


# ----------------------------------------------------------------------------
# Algorithm 3 / Theorem 2 written out (long double, small n)
# ----------------------------------------------------------------------------

def _solve_ld(Adense_ld, rhs_ld):
    """Partial-pivoting elimination in numpy long double (small systems)."""
    A = np.array(Adense_ld, dtype=np.longdouble)
    B = np.array(rhs_ld, dtype=np.longdouble)
    if B.ndim == 1:
        B = B[:, None]
    n = A.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0:
            raise ZeroDivisionError("singular")
        if p != k:
            A[[k, p]] = A[[p, k]]
            B[[k, p]] = B[[p, k]]
        m = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= np.outer(m, A[k, k:])
        B[k + 1:] -= np.outer(m, B[k])
    X = np.zeros_like(B)
    for i in range(n - 1, -1, -1):
        X[i] = (B[i] - A[i, i + 1:] @ X[i + 1:]) / A[i, i]
    return X


def z_vectors(a, b, k: int):
    """(Z^R_k, Z^L_k) of eq. z_vector for separator row k (0-based).

    B^R_k is the identity row at k followed by rows k+1..n-1 of A (restricted
    to columns k..n-1); B^L_k is rows 0..k-1 of A (columns 0..k) followed by an
    identity row at k (eq. matrixbrl with c_i = a_i).  Z^R_k solves
    B^R_k Z = e^R = (1, 0, ..., 0) on rows k..n-1, Z^L_k solves B^L_k Z = e^L =
    (0, ..., 0, 1) on rows 0..k.  Returned as long double arrays of the full
    length n, zero outside their support.
    """
    A = dense(a, b).astype(np.longdouble)
    n = A.shape[0]
    zr = np.zeros(n, dtype=np.longdouble)
    zl = np.zeros(n, dtype=np.longdouble)
    BR = A[k:, k:].copy()
    BR[0, :] = 0
    BR[0, 0] = 1
    eR = np.zeros(n - k, dtype=np.longdouble)
    eR[0] = 1
    zr[k:] = _solve_ld(BR, eR)[:, 0]
    BL = A[: k + 1, : k + 1].copy()
    BL[k, :] = 0
    BL[k, k] = 1
    eL = np.zeros(k + 1, dtype=np.longdouble)
    eL[k] = 1
    zl[: k + 1] = _solve_ld(BL, eL)[:, 0]
    return zr, zl


def dichotomy_ld(a, b, F, seps):
    """Algorithm 3 (separator values by Theorem 2) + Algorithm 1 (local solves).

    Rows are 0-based.  ``seps`` are the separator rows p_1 < ... < p_P, all in
    1..n-1; with p_0 = 0 and p_{P+1} = n the blocks are [p_{j-1}, p_j),
    j = 1..P+1, each starting at its left separator (the sums of eq. beta run
    over j = n_{i-1} .. n_i - 1).

      1.1  G_k = A^{-1} e_k for every separator k          (eq. green_v)
      1.2  Z^R_k, Z^L_k from eq. z_vector
      2.1  beta^R_j = sum_{i in block j} F_i G_{p_j}(i),
           beta^L_j = sum_{i in block j} F_i G_{p_{j-1}}(i)  (eq. beta_symn)
      2.2  x(p_i) = sum_{j <= i} beta^R_j Z^R_{p_j}(p_i)
                  + sum_{j >= i+1} beta^L_j Z^L_{p_{j-1}}(p_i)   (eq. theor_2)
      then every block interior is an independent Dirichlet problem with its
      two known end values (Lemma 1, Algorithm 1 step 3).
    Returns (X, x_sep) in long double; F has shape (n,) or (n, N).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    Fl = np.asarray(F, dtype=np.float64).astype(np.longdouble)
    squeeze = Fl.ndim == 1
    if squeeze:
        Fl = Fl[:, None]
    n, N = Fl.shape
    seps = [int(s) for s in seps]
    assert all(0 < s < n for s in seps) and seps == sorted(set(seps))
    P = len(seps)
    bounds = [0] + seps + [n]
    A = dense(a, b).astype(np.longdouble)
    # 1.1 inverse columns at the separators (A symmetric: also the rows)
    E = np.zeros((n, P), dtype=np.longdouble)
    for q, s in enumerate(seps):
        E[s, q] = 1
    G = _solve_ld(A, E) if P else np.zeros((n, 0), dtype=np.longdouble)
    # 1.2 homogeneous solutions
    Z = [z_vectors(a, b, s) for s in seps]
    # 2.1 beta per block (1-based block j = 1..P+1 -> python index j-1)
    betaR = {}
    betaL = {}
    for j in range(1, P + 2):
        lo, hi = bounds[j - 1], bounds[j]
        if j <= P:   # right separator p_j
            betaR[j] = (G[lo:hi, j - 1, None] * Fl[lo:hi]).sum(axis=0)
        if j >= 2:   # left separator p_{j-1}
            betaL[j] = (G[lo:hi, j - 2, None] * Fl[lo:hi]).sum(axis=0)
    # 2.2 separator values by Theorem 2
    xs = np.zeros((P, N), dtype=np.longdouble)
    for i in range(1, P + 1):
        acc = np.zeros(N, dtype=np.longdouble)
        for j in range(1, i + 1):
            acc += betaR[j] * Z[j - 1][0][seps[i - 1]]
        for j in range(i + 1, P + 2):
            acc += betaL[j] * Z[j - 2][1][seps[i - 1]]
        xs[i - 1] = acc
    # Algorithm 1 step 3: independent Dirichlet problems on block interiors
    X = np.zeros((n, N), dtype=np.longdouble)
    for q, s in enumerate(seps):
        X[s] = xs[q]
    known = set(seps)
    for j in range(1, P + 2):
        lo, hi = bounds[j - 1], bounds[j]
        rows = [r for r in range(lo, hi) if r not in known]
        if not rows:
            continue
        r0, r1 = rows[0], rows[-1] + 1
        Ai = A[r0:r1, r0:r1]
        rhs = Fl[r0:r1].copy()
        if r0 - 1 >= 0:
            rhs[0] -= A[r0, r0 - 1] * X[r0 - 1]
        if r1 < n:
            rhs[-1] -= A[r1 - 1, r1] * X[r1]
        X[r0:r1] = _solve_ld(Ai, rhs)
    return (X[:, 0] if squeeze else X), xs


def explicit_inverse(a, b):
    """A^{-1} from the explicit representation of Section 3.6 (eqs. x1-x3).

    For a symmetric matrix the products a_k / c_{k+1} in eq. x1 are all 1, so
    (A^{-1})_ij = y_i z_j for i <= j and z_i y_j for i >= j, where A Y = e_n
    and A Z = e_1 / y_1.  Y and Z come from the binary64 sweep.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    e_n = np.zeros(n)
    e_n[-1] = 1
    y = thomas_f64(a, b, e_n)
    e_1 = np.zeros(n)
    e_1[0] = 1.0 / y[0]
    z = thomas_f64(a, b, e_1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    # i <= j: y_i z_j;  i >= j: z_i y_j  -- both are y_min(i,j) * z_max(i,j)
    return y[np.minimum(i, j)] * z[np.maximum(i, j)]


def thomas_general(sub, diag, sup, F):
    """Textbook sweep in binary64 for a general tridiagonal matrix
    (A[i][i] = diag[i], A[i+1][i] = sub[i], A[i][i+1] = sup[i]), every column
    of F (shape (n,) or (n, N)); pure numpy, one row at a time."""
    sub, diag, sup = _f64(sub), _f64(diag), _f64(sup)
    F, squeeze = _as2d(F)
    n = diag.shape[0]
    X = np.array(F, dtype=np.float64, copy=True)
    d = np.empty(n)
    d[0] = diag[0]
    for i in range(1, n):           # forward elimination
        l = sub[i - 1] / d[i - 1]
        d[i] = diag[i] - l * sup[i - 1]
        X[i] -= l * X[i - 1]
    X[n - 1] /= d[n - 1]
    for i in range(n - 2, -1, -1):  # back substitution
        X[i] = (X[i] - sup[i] * X[i + 1]) / d[i]
    return X[:, 0] if squeeze else X


def symmetrizer(sub, sup):
    """t of the diagonal similarity of Section 3.5: with T = diag(t), T^{-1} A T
    is symmetric when sub[k] * sup[k] > 0; t_0 = 1, t_{k+1} = t_k sqrt(sub[k] / sup[k])."""
    sub, sup = _f64(sub), _f64(sup)
    t = np.ones(sub.shape[0] + 1)
    for k in range(sub.shape[0]):
        t[k + 1] = t[k] * np.sqrt(sub[k] / sup[k])
    return t


def algorithm2(a, b, F, ks):
    """Algorithm 2: the components k of every solution, X[k, :] = G_k^T F with
    A G_k = e_k (G_k by the binary64 sweep, then a plain matrix product).
    Returns an array of shape (len(ks), N)."""
    a, b = _f64(a), _f64(b)
    F, _ = _as2d(F)
    n = b.shape[0]
    ks = np.asarray(ks, dtype=np.int64)
    E = np.zeros((n, ks.size))
    E[ks, np.arange(ks.size)] = 1.0
    G = thomas_f64(a, b, E)          # columns G_k
    return G.T @ F
