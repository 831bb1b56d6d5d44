"""Pins of the Fourier Poisson oracle (Section 4a): the discrete solution of the
model problem in closed form, brute force on tiny meshes (the dense five-point
system), the library DST-I, the residual of the discrete equation, and planted
mistakes that these pins catch."""
import numpy as np
import pytest

from oracle import poisson as op


def _dense_laplacian(N1, N2, h1, h2):
    n1, n2 = N1 - 1, N2 - 1
    T1 = (np.diag(-2.0 * np.ones(n1)) + np.diag(np.ones(n1 - 1), 1) + np.diag(np.ones(n1 - 1), -1)) / h1 ** 2
    T2 = (np.diag(-2.0 * np.ones(n2)) + np.diag(np.ones(n2 - 1), 1) + np.diag(np.ones(n2 - 1), -1)) / h2 ** 2
    return np.kron(T1, np.eye(n2)) + np.kron(np.eye(n1), T2)   # index i * n2 + j


@pytest.mark.parametrize("N1,N2", [(8, 8), (16, 32), (64, 64), (33, 17)])
def test_model_problem_closed_form(N1, N2):
    f, u, h1, h2 = op.model_problem(N1, N2)
    got = op.fourier_poisson(f, h1, h2)
    assert np.max(np.abs(got - u)) <= 1e-12 * np.max(np.abs(u))


@pytest.mark.parametrize("N1,N2,h1,h2", [(6, 5, 0.2, 0.25), (9, 12, 1 / 9, 1 / 12), (12, 7, 0.05, 0.3)])
def test_brute_force_dense_system(N1, N2, h1, h2):
    rng = np.random.default_rng(N1 * 100 + N2)
    f = rng.standard_normal((N1 - 1, N2 - 1, 3))
    L = _dense_laplacian(N1, N2, h1, h2)
    ref = np.linalg.solve(-L, f.reshape(-1, 3)).reshape(f.shape)
    got = op.fourier_poisson(f, h1, h2)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_sine_basis_matches_library_dst1():
    scipy_fft = pytest.importorskip("scipy.fft")
    N2 = 21
    x = np.random.default_rng(1).standard_normal(N2 - 1)
    # scipy's DST-I: y_k = 2 sum_n x_n sin(pi (k+1)(n+1) / N2)
    assert np.allclose(2.0 * op.sine_matrix(N2) @ x, scipy_fft.dst(x, type=1), rtol=0, atol=1e-12)
    S = op.sine_matrix(N2)
    assert np.allclose(S @ S, (N2 / 2.0) * np.eye(N2 - 1), atol=1e-12)


def test_residual_of_the_discrete_equation():
    rng = np.random.default_rng(7)
    N1, N2, h1, h2 = 40, 24, 1 / 40, 1 / 24
    f = rng.standard_normal((N1 - 1, N2 - 1))
    u = op.fourier_poisson(f, h1, h2)
    assert np.max(np.abs(op.laplacian(u, h1, h2) + f)) <= 1e-9 * np.max(np.abs(f))


def test_planted_mistakes_are_caught(monkeypatch):
    N1, N2, h1, h2 = 9, 12, 1 / 9, 1 / 12
    f = np.random.default_rng(3).standard_normal((N1 - 1, N2 - 1))
    ref = np.linalg.solve(-_dense_laplacian(N1, N2, h1, h2), f.reshape(-1)).reshape(f.shape)
    good = op.mode_shifts
    for bad in (lambda *a: -good(*a), lambda N1, N2, h1, h2: good(N1, N2, h2, h1), lambda *a: 0.5 * good(*a)):
        monkeypatch.setattr(op, "mode_shifts", bad)
        assert np.max(np.abs(op.fourier_poisson(f, h1, h2) - ref)) > 1e-6 * np.max(np.abs(ref))
    monkeypatch.setattr(op, "mode_shifts", good)
    good_s = op.sine_matrix
    monkeypatch.setattr(op, "sine_matrix", lambda N2: good_s(N2 + 1)[:N2 - 1, :N2 - 1])
    assert np.max(np.abs(op.fourier_poisson(f, h1, h2) - ref)) > 1e-6 * np.max(np.abs(ref))
