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


# ---- alternating directions (Section 4b) ------------------------------------

@pytest.mark.parametrize("N,eps,n0", [(512, 1e-5, 17), (1024, 1e-5, 19), (64, 1e-3, 8)])
def test_adi_parameter_count_eq_ocenka1(N, eps, n0):
    # n0 = ceil(0.2 ln(4N/pi) ln(4/eps)), worked by hand: N=512: 0.2*6.480*12.899 = 16.72;
    # N=1024: 0.2*7.173*12.899 = 18.51; N=64, eps=1e-3: 0.2*4.401*8.294 = 7.30
    w = op.adi_parameters(N, eps)
    assert len(w) == n0
    h = 1.0 / N
    assert np.isclose(w[0], 4 / h ** 2 * np.sin(np.pi * h / 2) ** 2)
    assert np.isclose(w[-1], 4 / h ** 2 * np.cos(np.pi * h / 2) ** 2)
    assert np.allclose(w[1:] / w[:-1], w[1] / w[0])   # geometric


def test_adi_fixed_point_is_the_discrete_solution():
    # one Peaceman-Rachford step from the exact discrete solution returns it
    N = 24
    f, u, h1, h2 = op.model_problem(N, N)
    rng = np.random.default_rng(2)
    fr = rng.standard_normal((N - 1, N - 1))
    ur = op.fourier_poisson(fr, 1.0 / N, 1.0 / N)
    h = 1.0 / N
    for om in (3.0, 500.0):
        b = np.full(N - 1, 2.0 + om * h * h)
        a = -np.ones(N - 2)
        import oracle
        rhs = h * h * (om * ur + op._second_difference(ur, 1, h) + fr)
        uh = oracle.thomas_f64(a, b, rhs)
        assert np.max(np.abs(uh - ur)) <= 1e-11 * np.max(np.abs(ur))


@pytest.mark.parametrize("N", [32, 128])
def test_adi_reaches_eps_against_the_fourier_solution(N):
    eps = 1e-5
    f, u, _, _ = op.model_problem(N, N)
    got = op.peaceman_rachford(f, N, op.adi_parameters(N, eps))
    assert np.max(np.abs(got - u)) <= eps * np.max(np.abs(u))
    fr = np.random.default_rng(N).standard_normal((N - 1, N - 1, 2))
    ref = op.fourier_poisson(fr, 1.0 / N, 1.0 / N)
    got = op.peaceman_rachford(fr, N, op.adi_parameters(N, eps))
    assert np.max(np.abs(got - ref)) <= eps * np.max(np.abs(ref))
    # a planted mistake (omega scaled by h^2 twice) does not converge
    bad = op.peaceman_rachford(fr, N, op.adi_parameters(N, eps) / N ** 2)
    assert np.max(np.abs(bad - ref)) > 100 * eps * np.max(np.abs(ref))


def test_product_sine_transform_on_cpu():
    """The package's FFT-based type-I sine transform (plain torch, runs on CPU too)
    equals the oracle's explicit sine sums."""
    import torch
    from paper_0901_2859_gb300.poisson import dst1
    x = np.random.default_rng(11).standard_normal((4, 29, 3))
    got = dst1(torch.from_numpy(x), dim=1).numpy()
    ref = np.einsum("lj,ijn->iln", op.sine_matrix(30), x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    got0 = dst1(torch.from_numpy(x[:, :, 0].T.copy()), dim=0).numpy()
    assert np.allclose(got0, ref[:, :, 0].T, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
