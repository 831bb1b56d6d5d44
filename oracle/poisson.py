"""CPU oracle for the Poisson solvers of Section 4: variable separation (Fourier,
Section 4a) and alternating directions (Peaceman-Rachford, Section 4b).

TEST INFRASTRUCTURE ONLY: the tests and ``bench.py``'s CPU legs use this
module; the product path never imports it.  It shares no code with the
package's ``poisson`` module (which uses FFTs and the CUDA solves): the
transforms here are the explicit sine sums, the tridiagonal systems are the
oracle's binary64 sweep.

The problem (eq. poisson_difference on the mesh of eq. grid): on the mesh
x_i = i h1, y_j = j h2 of the rectangle [0, N1 h1] x [0, N2 h2], find u with
u = 0 on the boundary and, at the interior nodes 1 <= i <= N1-1,
1 <= j <= N2-1,

    (u[i+1,j] - 2u[i,j] + u[i-1,j]) / h1^2 + (u[i,j+1] - 2u[i,j] + u[i,j-1]) / h2^2 = -f[i,j].

Interior arrays are indexed [i-1, j-1] (shape (N1-1, N2-1)), with a trailing
axis for a series of right-hand sides f_n (eq. poisson_end).

Steps (Section 4a, eqs. fft_phi, SLAU_FFT):
  1. the sine coefficients along j:  f~_i(l) = (2/N2) sum_j f[i,j] sin(pi l j / N2),
     the inverse of the expansion f[i,j] = sum_l f~_i(l) sin(pi l j / N2);
  2. for every mode l, the tridiagonal system in i
         -u~_{i-1}(l) + (2 + d_l) u~_i(l) - u~_{i+1}(l) = h1^2 f~_i(l),
         d_l = 4 (h1/h2)^2 sin^2(pi l / (2 N2))          (eq. series_fft, sign flipped)
     with u~_0 = u~_{N1} = 0, solved by the sweep;
  3. the synthesis u[i,j] = sum_l u~_i(l) sin(pi l j / N2).

Pins (``tests/test_poisson_oracle.py``): the model problem of eq. poisson_test,
whose discrete solution is one eigenmode in closed form; brute force on tiny
meshes (the dense five-point system); scipy's DST-I; the discrete equation
itself (the residual of the oracle's u); for the alternating directions, the
parameter count of eq. ocenka1 worked by hand, the fixed point, and the
accuracy eps reached against the pinned Fourier solution.
"""
from __future__ import annotations

import numpy as np

from . import thomas_f64


def sine_matrix(N2: int) -> np.ndarray:
    """S[l-1, j-1] = sin(pi l j / N2) for 1 <= l, j <= N2-1 (the basis of eq. fft_phi),
    with the argument reduced exactly in integers: l j mod 2 N2."""
    idx = np.arange(1, N2, dtype=np.int64)
    k = np.outer(idx, idx) % (2 * N2)
    return np.sin(np.pi * k.astype(np.float64) / N2)


def mode_shifts(N1: int, N2: int, h1: float, h2: float) -> np.ndarray:
    """d_l = 4 (h1/h2)^2 sin^2(pi l / (2 N2)), l = 1..N2-1 (eq. series_fft)."""
    l = np.arange(1, N2, dtype=np.float64)
    return 4.0 * (h1 / h2) ** 2 * np.sin(np.pi * l / (2.0 * N2)) ** 2


def fourier_poisson(f, h1: float, h2: float) -> np.ndarray:
    """u at the interior nodes for f of shape (N1-1, N2-1) or (N1-1, N2-1, N)."""
    f = np.asarray(f, dtype=np.float64)
    series = f.ndim == 3
    if not series:
        f = f[:, :, None]
    n1, n2, N = f.shape
    N1, N2 = n1 + 1, n2 + 1
    S = sine_matrix(N2)
    # step 1: coefficients f~[l, i, n]
    ft = (2.0 / N2) * np.einsum("lj,ijn->lin", S, f)
    d = mode_shifts(N1, N2, h1, h2)
    ut = np.empty_like(ft)
    a = -np.ones(n1 - 1)
    for l in range(n2):   # step 2: one series per mode (eq. poisson_end)
        b = np.full(n1, 2.0 + d[l])
        ut[l] = thomas_f64(a, b, h1 * h1 * ft[l])
    u = np.einsum("lj,lin->ijn", S, ut)   # step 3
    return u if series else u[:, :, 0]


def laplacian(u, h1: float, h2: float) -> np.ndarray:
    """The five-point operator of eq. poisson_difference at the interior nodes,
    u extended by zeros on the boundary."""
    u = np.asarray(u, dtype=np.float64)
    pad = [(1, 1), (1, 1)] + [(0, 0)] * (u.ndim - 2)
    U = np.pad(u, pad)
    return ((U[2:, 1:-1] - 2 * U[1:-1, 1:-1] + U[:-2, 1:-1]) / h1 ** 2 +
            (U[1:-1, 2:] - 2 * U[1:-1, 1:-1] + U[1:-1, :-2]) / h2 ** 2)


def model_problem(N1: int, N2: int):
    """Eq. poisson_test on the unit square (h1 = 1/N1, h2 = 1/N2):
    f = 8 pi^2 sin(2 pi x) sin(2 pi y), and the exact solution of the discrete
    equation.  sin(2 pi x_i) is an eigenvector of the second difference with
    eigenvalue -(4/h^2) sin^2(pi h), so u = f / ((4/h1^2) sin^2(pi h1) + (4/h2^2) sin^2(pi h2)).
    Returns (f, u, h1, h2) at the interior nodes."""
    h1, h2 = 1.0 / N1, 1.0 / N2
    i = np.arange(1, N1, dtype=np.int64)
    j = np.arange(1, N2, dtype=np.int64)
    sx = np.sin(np.pi * ((2 * i) % (2 * N1)).astype(np.float64) / N1)   # sin(2 pi i / N1)
    sy = np.sin(np.pi * ((2 * j) % (2 * N2)).astype(np.float64) / N2)
    f = 8.0 * np.pi ** 2 * np.outer(sx, sy)
    lam = 4.0 / h1 ** 2 * np.sin(np.pi * h1) ** 2 + 4.0 / h2 ** 2 * np.sin(np.pi * h2) ** 2
    return f, f / lam, h1, h2


# --------------------------------------------------------------------------
# Alternating directions (Section 4b): the Peaceman-Rachford iteration
# (eqs. adi_iter, adi_iter2) on the square mesh N1 = N2 = N, h = 1/N.
#
# Readings (the paper leaves them open):
#  * sign: the iteration relaxes du/dt = Lambda u + f, whose steady state is
#    the discrete problem Lambda u = -f of eq. poisson_difference;
#  * parameters: omega_k = 1/tau_k (tau^(1) = tau^(2)), a geometric sequence
#    over the spectrum [delta, Delta] of -Lambda_alpha, delta = (4/h^2)
#    sin^2(pi h / 2), Delta = (4/h^2) cos^2(pi h / 2), endpoints included;
#  * their number n_0(eps) = ceil(0.2 ln(4N/pi) ln(4/eps)) (eq. ocenka1),
#    applied once each from u = 0.
# --------------------------------------------------------------------------

def adi_parameters(N: int, eps: float) -> np.ndarray:
    """omega_1..omega_{n0} for the N x N mesh and accuracy eps."""
    h = 1.0 / N
    lo = 4.0 / h ** 2 * np.sin(np.pi * h / 2.0) ** 2
    hi = 4.0 / h ** 2 * np.cos(np.pi * h / 2.0) ** 2
    n0 = int(np.ceil(0.2 * np.log(4.0 * N / np.pi) * np.log(4.0 / eps)))
    k = np.arange(n0, dtype=np.float64)
    return lo * (hi / lo) ** (k / max(n0 - 1, 1))


def _second_difference(u, axis: int, h: float) -> np.ndarray:
    pad = [(0, 0)] * u.ndim
    pad[axis] = (1, 1)
    U = np.pad(u, pad)
    sl = lambda a, b: tuple(slice(a, b) if d == axis else slice(None) for d in range(u.ndim))
    return (U[sl(2, None)] - 2.0 * U[sl(1, -1)] + U[sl(None, -2)]) / h ** 2


def peaceman_rachford(f, N: int, omegas) -> np.ndarray:
    """u after one pass over `omegas`, from u = 0; f of shape (N-1, N-1) or (N-1, N-1, S).
    Each step solves (omega I - Lambda_1) u' = (omega I + Lambda_2) u + f along i, then
    (omega I - Lambda_2) u'' = (omega I + Lambda_1) u' + f along j, scaled by h^2 into
    tridiag(-1, 2 + omega h^2, -1) systems solved by the sweep."""
    f = np.asarray(f, dtype=np.float64)
    series = f.ndim == 3
    if not series:
        f = f[:, :, None]
    n, _, S = f.shape
    h = 1.0 / N
    u = np.zeros_like(f)
    a = -np.ones(n - 1)
    for om in omegas:
        b = np.full(n, 2.0 + om * h * h)
        rhs = h * h * (om * u + _second_difference(u, 1, h) + f)         # along i; columns (j, s)
        uh = thomas_f64(a, b, rhs.reshape(n, n * S)).reshape(n, n, S)
        rhs = h * h * (om * uh + _second_difference(uh, 0, h) + f)       # along j; columns (i, s)
        rt = np.ascontiguousarray(rhs.transpose(1, 0, 2)).reshape(n, n * S)
        u = thomas_f64(a, b, rt).reshape(n, n, S).transpose(1, 0, 2)
    u = np.ascontiguousarray(u)
    return u if series else u[:, :, 0]
