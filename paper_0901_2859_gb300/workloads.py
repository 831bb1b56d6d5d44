"""Seeded synthetic workloads shaped like the paper's series of tridiagonal systems.

This module only draws inputs (matrices a, b and right-hand sides F, W); it
holds none of the solver's arithmetic, and both the CUDA path and the CPU
oracle consume exactly what it returns.  All generators use numpy's PCG64
(``numpy.random.default_rng(seed)``) on the host in binary64 and cast at the
end, so a (config, seed) pair always gives the same bytes.

Workloads (sizes are the defaults; every generator takes smaller sizes too):

``plain_fp64``   n = 1024, a_i ~ U[-1, -0.5], b_i ~ U[2.5, 3.5] (strictly
                 diagonally dominant), N = 64, F ~ N(0, 1), binary64.
``poisson2d``    the 1D -u'' + s u stencil of the Fourier-mode systems of
                 Section 4: a_i = -1, b_i = 2 + s, s = 4 sin^2(pi / (2 (n+1))),
                 n = 4096, N = 4096.  Columns 0..63 are pure sine modes
                 sin(pi k i / (n+1)) with k in {1, 2, 3, n/2, n-1, n} plus
                 uniform random k; the other columns are a mode with random k
                 plus N(0, 1) noise.
``precision``    n = 16384, N = 8192, a_i = -1, b_i = 2 + s with
                 s = 10^U[-6, 0] drawn per seed, F ~ N(0, 1) in binary32.
``batching``     512 matrices of Fourier modes m = 1..512 of a K = 512 grid:
                 a_i = -1, b_i = 2 + 4 sin^2(pi m / (2 (K+1))); sizes
                 ln n ~ N(ln 2048, 1) rounded and clipped to [256, 65536];
                 N_m ~ U{1..2048}; F ~ N(0, 1) in binary32.
``diff``         n = 8192, N = 2048, a_i ~ U[-1, -0.5], b_i ~ U[2.2, 3.0],
                 F, W ~ N(0, 1) in binary32 (loss = sum(W * X)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Series:
    """One constant matrix with its block of right-hand sides."""
    a: np.ndarray            # (n-1,) off-diagonal, binary64
    b: np.ndarray            # (n,) diagonal, binary64
    F: np.ndarray            # (n, N) right-hand sides, RHS contiguous
    W: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.b.shape[0])

    @property
    def N(self) -> int:
        return int(self.F.shape[1])


def _modes(n: int, ks: np.ndarray) -> np.ndarray:
    """sin(pi k i / (n+1)), i = 1..n, with the argument reduced exactly in integers."""
    i = np.arange(1, n + 1, dtype=np.int64)
    m = np.outer(i, np.asarray(ks, dtype=np.int64)) % (2 * (n + 1))
    return np.sin(np.pi * m.astype(np.float64) / (n + 1))


def plain_fp64(seed: int = 0, n: int = 1024, N: int = 64) -> Series:
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, -0.5, n - 1)
    b = rng.uniform(2.5, 3.5, n)
    F = rng.standard_normal((n, N))
    return Series(a, b, F, meta={"workload": "plain_fp64", "seed": seed, "M": 8})


def poisson_shift(n: int) -> float:
    return float(4.0 * np.sin(np.pi / (2.0 * (n + 1))) ** 2)


def poisson2d(seed: int = 0, n: int = 4096, N: int = 4096, dtype=np.float64) -> Series:
    rng = np.random.default_rng(seed)
    s = poisson_shift(n)
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + s)
    n_pure = min(64, N)
    fixed = [k for k in (1, 2, 3, n // 2, n - 1, n) if 1 <= k <= n]
    ks_pure = np.array((fixed + list(rng.integers(1, n + 1, size=max(0, n_pure - len(fixed)))))[:n_pure])
    F = np.empty((n, N))
    F[:, :n_pure] = _modes(n, ks_pure)
    if N > n_pure:
        ks = rng.integers(1, n + 1, size=N - n_pure)
        F[:, n_pure:] = _modes(n, ks) + rng.standard_normal((n, N - n_pure))
    return Series(a, b, F.astype(dtype), meta={"workload": "poisson2d", "seed": seed, "s": s,
                                               "pure_modes": ks_pure.tolist()})


def precision(seed: int = 0, n: int = 16384, N: int = 8192, s: float | None = None,
              dtype=np.float32) -> Series:
    rng = np.random.default_rng(seed)
    if s is None:
        s = float(10.0 ** rng.uniform(-6.0, 0.0))
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + s)
    F = rng.standard_normal((n, N), dtype=np.float32 if dtype == np.float32 else np.float64)
    return Series(a, b, F.astype(dtype, copy=False), meta={"workload": "precision", "seed": seed, "s": s})


def batching(seed: int = 0, count: int = 512, K: int = 512, n_median: int = 2048,
             n_min: int = 256, n_max: int = 65536, N_max: int = 2048,
             rhs: bool = True) -> list[Series]:
    """Fourier-mode series of a K-mode grid; rhs=False skips drawing F (sizes only)."""
    rng = np.random.default_rng(seed)
    ns = np.clip(np.rint(np.exp(rng.normal(np.log(n_median), 1.0, size=count))), n_min, n_max).astype(np.int64)
    Ns = rng.integers(1, N_max + 1, size=count)
    out = []
    for m in range(count):
        n, N = int(ns[m]), int(Ns[m])
        mode = m + 1
        s = float(4.0 * np.sin(np.pi * mode / (2.0 * (K + 1))) ** 2)
        a = -np.ones(n - 1)
        b = np.full(n, 2.0 + s)
        F = rng.standard_normal((n, N), dtype=np.float32) if rhs else np.empty((n, 0), np.float32)
        out.append(Series(a, b, F, meta={"workload": "batching", "mode": mode, "s": s, "N": N}))
    return out


def diff(seed: int = 0, n: int = 8192, N: int = 2048) -> Series:
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, -0.5, n - 1)
    b = rng.uniform(2.2, 3.0, n)
    F = rng.standard_normal((n, N), dtype=np.float32)
    W = rng.standard_normal((n, N), dtype=np.float32)
    return Series(a, b, F, W, meta={"workload": "diff", "seed": seed})


def random_dominant(seed: int, n: int, N: int, dtype=np.float64, margin: float = 0.5) -> Series:
    """Small general test systems: a_i ~ U[-1, 1], b_i = +-(|a_{i-1}| + |a_i| + U[margin, margin+1])."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, max(n - 1, 0))
    pad = np.r_[0.0, np.abs(a)] + np.r_[np.abs(a), 0.0]
    b = (pad + rng.uniform(margin, margin + 1.0, n)) * rng.choice([-1.0, 1.0], size=n)
    F = rng.standard_normal((n, N)).astype(dtype)
    return Series(a, b, F, meta={"workload": "random_dominant", "seed": seed})
