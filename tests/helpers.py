"""Shared test helpers (no solver arithmetic)."""
import numpy as np

U64 = np.finfo(np.float64).eps / 2


def relerr(x, ref):
    """max over columns of max_i |x - ref| / max_i |ref| (relative max-norm per column)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    den = np.maximum(np.max(np.abs(ref), axis=0), np.finfo(np.float64).tiny)
    return float(np.max(np.max(np.abs(x - ref), axis=0) / den)) if x.size else 0.0


def kappa_inf_estimate(a, b):
    """kappa_inf of the shifted-Laplacian-like matrices used here (upper bound by Gershgorin/eigs)."""
    import oracle
    n = len(b)
    if n <= 2000:
        A = oracle.dense(a, b)
        return float(np.linalg.cond(A, p=np.inf))
    Ainv_col = oracle.solve_hi(a, b, np.ones(n))     # A^{-1} 1 bounds ||A^{-1}||_inf for M-matrices
    normA = np.max(np.abs(b) + np.r_[np.abs(a), 0] + np.r_[0, np.abs(a)])
    return float(normA * np.max(np.abs(Ainv_col)))
