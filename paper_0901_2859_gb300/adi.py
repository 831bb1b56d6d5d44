"""Series of Poisson problems by alternating directions (Section 4b).

The Peaceman-Rachford iteration (eqs. adi_iter, adi_iter2) on the square mesh
N1 = N2 = N, h = 1/N, u = 0 on the boundary, for the five-point problem
Lambda u = -f (eq. poisson_difference), Lambda = Lambda_1 + Lambda_2
(eq. operator2).  Each iteration k with parameter omega_k = 1/tau_k takes two
half steps,

    (omega I - Lambda_1) u' = (omega I + Lambda_2) u + f     (along i, every j)
    (omega I - Lambda_2) u  = (omega I + Lambda_1) u' + f    (along j, every i)

and, scaled by h^2, every half step is a series of tridiagonal systems with
the one matrix tridiag(-1, 2 + omega h^2, -1) (the matrices C^(1), C^(2) of
the paper, sign flipped): the grid lines are the right-hand sides.  The n_0
parameters are cyclic, so one plan per parameter serves every iteration and
both directions (the paper's point: only n_0 preparations).

Parameters (the paper defers their choice to the literature): a geometric
sequence over the spectrum [delta, Delta] of -Lambda_alpha, delta =
(4/h^2) sin^2(pi h/2), Delta = (4/h^2) cos^2(pi h/2), endpoints included,
n_0(eps) = ceil(0.2 ln(4N/pi) ln(4/eps)) of them (eq. ocenka1), applied once
each from u = 0.

Arrays hold the interior nodes [i-1, j-1]: shape (N-1, N-1), or
(N-1, N-1, S) for a series of S problems solved together.

Precision: ``"fp32"`` keeps u in binary32 and solves in binary32. It is the
fastest, but the binary32 solves of the small-omega systems (condition up to
about 4 / (pi h)^2) leave an error of order 1e-5 at N = 256. ``"fp32_refined"``
keeps u in binary64 and solves binary32 right-hand sides to binary64 results.
``"fp64"`` is binary64 throughout.  The half steps' right-hand sides (a
three-point difference along the lines, and a transpose every second half
step) are formed in one pass by the library's ``tdm_adi_rhs`` kernel; the
tridiagonal series go through its dichotomy solve.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib
from .api import _stream_ptr, check, prepare

__all__ = ["PeacemanRachford", "adi_parameters"]


def adi_parameters(N: int, eps: float) -> np.ndarray:
    """omega_k, k = 1..n_0(eps), for the N x N mesh (see the module docstring)."""
    if N < 2 or not (0.0 < eps < 1.0):
        raise ValueError("need N >= 2 and 0 < eps < 1")
    h = 1.0 / N
    lo = 4.0 / (h * h) * math.sin(math.pi * h / 2.0) ** 2
    hi = 4.0 / (h * h) * math.cos(math.pi * h / 2.0) ** 2
    n0 = math.ceil(0.2 * math.log(4.0 * N / math.pi) * math.log(4.0 / eps))
    return np.array([lo * (hi / lo) ** (k / max(n0 - 1, 1)) for k in range(n0)])


class PeacemanRachford:
    """One prepared plan per parameter; ``solve`` runs n_0 iterations."""

    def __init__(self, N: int, eps: float = 1e-5, precision: str = "fp32", device=None):
        if precision not in ("fp32", "fp32_refined", "fp64"):
            raise ValueError("precision must be 'fp32', 'fp32_refined' or 'fp64'")
        self.N, self.eps, self.precision = int(N), float(eps), precision
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.omegas = adi_parameters(self.N, self.eps)
        n, h = self.N - 1, 1.0 / self.N
        a = np.full(max(n - 1, 0), -1.0)
        self.plans = [prepare(a, np.full(n, 2.0 + om * h * h), device=self.device) for om in self.omegas]

    def close(self) -> None:
        for p in self.plans:
            p.close()
        self.plans = []

    def _rhs(self, v: torch.Tensor, f: torch.Tensor, om: float, buf: torch.Tensor) -> None:
        """buf[a, (b, s)] = h^2 (omega v + Lambda_b v + f) = (omega h^2 - 2) v + h^2 f
        + the neighbours along b (u = 0 beyond the ends), formed in one pass into the
        solver's layout and precision by ``tdm_adi_rhs``; v and f may be transposed views."""
        n, _, S = v.shape
        h2 = 1.0 / (self.N * self.N)
        if f.dtype != v.dtype or f.shape != v.shape:
            raise ValueError("v and f must have one dtype and shape")
        if v.stride(2) != 1 or f.stride(2) != 1:
            v, f = v.contiguous(), f.contiguous()
        st = _lib.load().tdm_adi_rhs(
            ctypes.c_void_p(v.data_ptr()), v.stride(0), v.stride(1), ctypes.c_void_p(f.data_ptr()), f.stride(0),
            f.stride(1), n, n, S, om * h2 - 2.0, h2, int(v.dtype == torch.float64), ctypes.c_void_p(buf.data_ptr()),
            buf.stride(0), int(buf.dtype == torch.float64), _stream_ptr(buf.device))
        check(st, "tdm_adi_rhs")

    def _half_step(self, plan, v: torch.Tensor, f: torch.Tensor, om: float, buf: torch.Tensor) -> torch.Tensor:
        """v, f in the layout [a, b, s]: a the axis the systems run along, b the
        lines (their right-hand sides), s the problem.  Returns w, [a, b, s], with
        tridiag(-1, 2 + omega h^2, -1) w = h^2 (omega v + Lambda_b v + f) along a."""
        n, _, S = v.shape
        self._rhs(v, f, om, buf)
        w = torch.empty(buf.shape, dtype=v.dtype, device=buf.device)
        plan.solve(buf[:, :n * S], self.precision, out=w[:, :n * S])
        return w[:, :n * S].view(n, n, S)

    def solve(self, f: torch.Tensor) -> torch.Tensor:
        n = self.N - 1
        if f.shape[:2] != (n, n) or f.ndim not in (2, 3):
            raise ValueError(f"f must have shape ({n}, {n}) or ({n}, {n}, S)")
        dt = torch.float32 if self.precision == "fp32" else torch.float64          # u and f
        dt_in = torch.float64 if self.precision == "fp64" else torch.float32       # the solves' right-hand sides
        series = f.ndim == 3
        f = f.to(device=self.device, dtype=dt)
        if not series:
            f = f[:, :, None]
        S = f.shape[2]
        ld = (n * S + 3) // 4 * 4   # a row pitch of 16-byte multiples keeps the tiles TMA-staged
        buf = torch.empty((n, ld), dtype=dt_in, device=self.device)
        u = torch.zeros((n, n, S), dtype=dt, device=self.device)   # [i, j, s]
        fT = f.transpose(0, 1)                                        # [j, i, s]
        for plan, om in zip(self.plans, self.omegas):
            uh = self._half_step(plan, u, f, float(om), buf)                               # along i: [i, j, s]
            u = self._half_step(plan, uh.transpose(0, 1), fT, float(om), buf).transpose(0, 1)   # along j
        u = u.contiguous()
        return u if series else u[:, :, 0]
