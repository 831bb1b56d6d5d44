"""Series of Poisson problems by variable separation (Section 4a).

On the mesh x_i = i h1, y_j = j h2 (eq. grid) with u = 0 on the boundary,
``FourierPoisson`` solves the five-point equation (eq. poisson_difference)

    (u[i+1,j] - 2u[i,j] + u[i-1,j]) / h1^2 + (u[i,j+1] - 2u[i,j] + u[i,j-1]) / h2^2 = -f_n[i,j]

for a series of right-hand sides f_n at once:

  1. the sine coefficients of every f_n along j (the inverse of eq. fft_phi),
     a type-I discrete sine transform computed with a real FFT of the odd
     extension (cuFFT through ``torch.fft``; the transform is the FFT the
     paper prescribes for these sums);
  2. for every mode l, the series B_l u_n(l) = g_n(l) of eq. poisson_end with
     B_l = tridiag(-1, 2 + d_l, -1), d_l = 4 (h1/h2)^2 sin^2(pi l / (2 N2))
     (eq. series_fft with the sign flipped, so that B_l is positive
     definite): one prepared plan per mode, all modes in one batched call of
     the dichotomy solver;
  3. the synthesis of eq. fft_phi, the same transform.

Arrays hold the interior nodes, [i-1, j-1], shape (N1-1, N2-1) or
(N1-1, N2-1, N) for a series of N problems.

Precision: ``"fp64"`` runs the binary64 dichotomy (one launch per mode);
``"fp32_refined"`` runs the binary32 solve with refinement to binary64
results (one launch per tile shape).  With binary64 right-hand sides the
refined path solves each as the sum of two binary32 parts, f = hi + lo
(``rhs_split``, default on), so that the result keeps binary64 accuracy.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .api import prepare, solve_batched

__all__ = ["FourierPoisson", "dst1"]


def dst1(x: torch.Tensor, dim: int) -> torch.Tensor:
    """y_l = sum_{j=1}^{M} x_j sin(pi l j / (M+1)), l = 1..M, along `dim`
    (M = x.shape[dim]), via the FFT of the odd extension of length 2(M+1):
    its coefficient l is -2i y_l."""
    x = x.movedim(dim, -1)
    M = x.shape[-1]
    z = torch.zeros(x.shape[:-1] + (1,), dtype=x.dtype, device=x.device)
    ext = torch.cat([z, x, z, -x.flip(-1)], dim=-1)
    y = -0.5 * torch.fft.rfft(ext, dim=-1).imag[..., 1:M + 1]
    return y.movedim(-1, dim)


class FourierPoisson:
    """Prepared mode matrices for an (N1 x N2)-step mesh; ``solve`` takes f_n."""

    def __init__(self, N1: int, N2: int, h1: float | None = None, h2: float | None = None,
                 precision: str = "fp32_refined", device=None, rhs_split: bool = True, block_rows: int = 0):
        if N1 < 2 or N2 < 2:
            raise ValueError("the mesh needs at least one interior node in each direction")
        if precision not in ("fp64", "fp32_refined"):
            raise ValueError("precision must be 'fp64' or 'fp32_refined'")
        self.N1, self.N2 = int(N1), int(N2)
        self.h1 = float(h1) if h1 is not None else 1.0 / N1
        self.h2 = float(h2) if h2 is not None else 1.0 / N2
        self.precision = precision
        self.rhs_split = rhs_split
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        n1, n2 = self.N1 - 1, self.N2 - 1
        l = np.arange(1, n2 + 1, dtype=np.float64)
        self.d = 4.0 * (self.h1 / self.h2) ** 2 * np.sin(np.pi * l / (2.0 * self.N2)) ** 2   # eq. series_fft
        a = np.full(max(n1 - 1, 0), -1.0)
        self.plans = [prepare(a, np.full(n1, 2.0 + dl), block_rows=block_rows, device=self.device) for dl in self.d]

    def close(self) -> None:
        for p in self.plans:
            p.close()
        self.plans = []

    def solve(self, f: torch.Tensor, events: list | None = None) -> torch.Tensor:
        """u for f; with `events` (a list), CUDA events are appended after the
        analysis, the mode solves and the synthesis (after one at the start)."""
        n1, n2 = self.N1 - 1, self.N2 - 1

        def mark():
            if events is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                events.append(e)
        if f.shape[:2] != (n1, n2) or f.ndim not in (2, 3):
            raise ValueError(f"f must have shape ({n1}, {n2}) or ({n1}, {n2}, N)")
        series = f.ndim == 3
        f = f.to(device=self.device, dtype=torch.float64)
        if not series:
            f = f[:, :, None]
        N = f.shape[2]
        mark()
        # 1. g[l, i, n] = h1^2 f~_i(l), f~ = (2/N2) sum_j f[i,j] sin(pi l j / N2)
        g = dst1(f, dim=1).permute(1, 0, 2).mul_(2.0 * self.h1 * self.h1 / self.N2)
        mark()
        # 2. one series per mode; every mode's block starts 16-byte aligned (row
        # pitch a multiple of 4 elements), as the solver requires
        split = self.precision == "fp32_refined" and self.rhs_split
        cols = 2 * N if split else N
        ld = (cols + 3) // 4 * 4
        if self.precision == "fp64":
            F = torch.empty((n2, n1, ld), dtype=torch.float64, device=self.device)
            F[:, :, :N] = g
        else:
            F = torch.empty((n2, n1, ld), dtype=torch.float32, device=self.device)
            F[:, :, :N] = g
            if split:   # f = hi + lo, both binary32; the solves are linear
                F[:, :, N:2 * N] = g - F[:, :, :N].to(torch.float64)
        X = torch.empty((n2, n1, ld), dtype=torch.float64, device=self.device)
        solve_batched(self.plans, [F[l, :, :cols] for l in range(n2)], self.precision,
                      outs=[X[l, :, :cols] for l in range(n2)])
        ut = X[:, :, :N] + X[:, :, N:2 * N] if split else X[:, :, :N]
        mark()
        # 3. u[i, j, n] = sum_l u~_i(l) sin(pi l j / N2)
        u = dst1(ut.permute(1, 0, 2), dim=1)
        mark()
        return u if series else u[:, :, 0]

    @staticmethod
    def model_rhs(N1: int, N2: int, device=None) -> torch.Tensor:
        """f = 8 pi^2 sin(2 pi x) sin(2 pi y) at the interior nodes of the unit
        square (the model problem of eq. poisson_test)."""
        i = torch.arange(1, N1, dtype=torch.float64, device=device)
        j = torch.arange(1, N2, dtype=torch.float64, device=device)
        return 8.0 * math.pi ** 2 * torch.outer(torch.sin(2 * math.pi * i / N1), torch.sin(2 * math.pi * j / N2))
