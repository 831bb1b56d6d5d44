"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each compares the oracle with an
independent source -- a library routine (LAPACK via numpy/scipy), a closed
form, the worked example of Section 3.5, an identity of the paper (Lemma 2,
Theorem 2, Theorem 4, the explicit inverse of Section 3.6), central finite
differences -- and the planted-mistake tests show that each pin fails when a
plausible mistake (a sign, a dropped term, a shifted index) is put into the
oracle's inputs.
"""
import os

import numpy as np
import pytest

U64 = np.finfo(np.float64).eps / 2


def _dominant(rng, n, lo=2.5, hi=3.5, alo=-1.0, ahi=-0.5):
    return rng.uniform(alo, ahi, n - 1), rng.uniform(lo, hi, n)


def _rel(x, ref):
    x, ref = np.atleast_2d(np.asarray(x, float).T).T, np.atleast_2d(np.asarray(ref, float).T).T
    return float(np.max(np.max(np.abs(x - ref), axis=0) / np.maximum(np.max(np.abs(ref), axis=0), 1e-300)))


# --------------------------------------------------------------------------
# library-routine pins
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 7, 33, 64])
def test_gauss_ld_matches_lapack_on_general_matrices(oracle, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
    F = rng.standard_normal((n, 4))
    X = oracle.gauss_ld(A, F)
    ref = np.linalg.solve(A, F)
    cond = np.linalg.cond(A)
    assert _rel(X, ref) <= 50 * cond * U64


@pytest.mark.parametrize("n", [1, 2, 3, 7, 33, 64])
def test_thomas_matches_gauss_ld(oracle, n):
    rng = np.random.default_rng(100 + n)
    a, b = _dominant(rng, n)
    F = rng.standard_normal((n, 5))
    X = oracle.thomas_f64(a, b, F)
    ref = oracle.gauss_ld(oracle.dense(a, b), F)
    assert _rel(X, ref) <= 1e-14


@pytest.mark.parametrize("n,s", [(200, 1.0), (2000, 1e-4), (4096, 5.88e-7)])
def test_solve_hi_matches_scipy_banded(oracle, n, s):
    from scipy.linalg import solve_banded
    rng = np.random.default_rng(7)
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + s)
    F = rng.standard_normal((n, 3))
    ab = np.zeros((3, n))
    ab[0, 1:] = a
    ab[1] = b
    ab[2, :-1] = a
    ref = solve_banded((1, 1), ab, F)
    X = oracle.solve_hi(a, b, F)
    kappa = np.linalg.cond(oracle.dense(a, b)) if n <= 2000 else 4.0 / (s + (np.pi / (n + 1)) ** 2)
    # LAPACK's banded LU is only accurate to ~kappa*u; the oracle must agree within that
    assert _rel(X, ref) <= 10 * kappa * U64


# --------------------------------------------------------------------------
# closed forms (Section 4: sine modes of the second-difference operator)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [64, 1024, 4096])
@pytest.mark.parametrize("s", [1.0, 1e-3, 5.88e-7])
def test_solve_hi_matches_eigen_closed_form(oracle, n, s):
    ks = sorted({1, 2, 3, n // 2, n - 1, n})
    F, X, lam = oracle.eigen_closed_form(n, 2.0 + s, ks)
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + s)
    got = oracle.solve_hi(a, b, F)
    lam_min = lam.min()
    for c, k in enumerate(ks):
        tol = max(1e-13, 10 * U64 * lam[c] / lam_min)
        assert _rel(got[:, c], X[:, c]) <= tol, (k, _rel(got[:, c], X[:, c]), tol)


def test_eigenvalues_match_lapack(oracle):
    n, s = 48, 1e-3
    _, _, lam = oracle.eigen_closed_form(n, 2.0 + s, np.arange(1, n + 1))
    ref = np.linalg.eigvalsh(oracle.dense(-np.ones(n - 1), np.full(n, 2.0 + s)))
    assert np.max(np.abs(np.sort(lam) - ref)) <= 1e-14


# --------------------------------------------------------------------------
# identities of the paper
# --------------------------------------------------------------------------

def test_lemma2_inverse_is_symmetric(oracle):
    """Lemma 2: G_k = A^{-1} e_k is both column and row k of A^{-1}."""
    rng = np.random.default_rng(3)
    n = 300
    a, b = _dominant(rng, n, 2.2, 3.0)
    Ainv = oracle.solve_hi(a, b, np.eye(n))
    scale = np.abs(Ainv).max()
    assert np.max(np.abs(Ainv - Ainv.T)) <= 1e-15 * scale * 10


def test_explicit_inverse_section_3_6(oracle):
    rng = np.random.default_rng(4)
    n = 40
    a, b = _dominant(rng, n)
    Ainv = oracle.explicit_inverse(a, b)
    ref = oracle.gauss_ld(oracle.dense(a, b), np.eye(n))
    assert np.max(np.abs(Ainv - ref)) <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("seps", [[], [1], [5], [1, 2, 3], [4, 9, 10, 17, 30], list(range(1, 39, 2)), [38]])
def test_theorem2_dichotomy_reaches_the_definition(oracle, seps):
    """Theorem 2 + Lemma 1: Algorithm 3 followed by local solves equals A^{-1} F."""
    rng = np.random.default_rng(len(seps))
    n = 39
    a, b = _dominant(rng, n)
    F = rng.standard_normal((n, 3))
    X, xs = oracle.dichotomy_ld(a, b, F, seps)
    ref = oracle.gauss_ld(oracle.dense(a, b), F)
    assert _rel(np.asarray(X, float), ref) <= 1e-15
    if seps:
        assert _rel(np.asarray(xs, float), ref[seps]) <= 1e-15


def test_theorem2_holds_without_dominance(oracle):
    """Theorem 2 needs only a nondegenerate A (and nonsingular B^R, B^L)."""
    rng = np.random.default_rng(11)
    n = 24
    a = rng.uniform(-1, 1, n - 1)
    b = rng.uniform(-1, 1, n)
    F = rng.standard_normal((n, 2))
    X, _ = oracle.dichotomy_ld(a, b, F, [6, 12, 18])
    ref = oracle.gauss_ld(oracle.dense(a, b), F)
    assert _rel(np.asarray(X, float), ref) <= 1e-11


@pytest.mark.parametrize("n,lo,hi", [(40, 2.0, 2.0), (40, 2.2, 3.0), (40, 2.5, 3.5)])
def test_theorem4_z_bounded_under_dominance(oracle, n, lo, hi):
    """Theorem 4: diagonal dominance (one row strict) gives ||Z^{R,L}||_C <= 1."""
    rng = np.random.default_rng(5)
    a = -np.ones(n - 1)
    b = rng.uniform(lo, hi, n)
    b[0] = max(b[0], 1.5)        # first row strictly dominant
    for k in (1, 7, 20, 38):
        zr, zl = oracle.z_vectors(a, b, k)
        assert np.max(np.abs(zr)) <= 1 + 1e-15 and np.max(np.abs(zl)) <= 1 + 1e-15
        assert zr[k] == 1 and zl[k] == 1


def test_theorem4_bound_can_fail_without_dominance(oracle):
    n = 20
    a = -np.ones(n - 1)
    b = np.full(n, 1.9)          # |b| < |a_{i-1}| + |a_i|: not dominant
    zr, zl = oracle.z_vectors(a, b, 10)
    assert max(np.max(np.abs(zr)), np.max(np.abs(zl))) > 1


def test_omega_levels_worked_example():
    """Section 3.5: p = 15 gives Omega_1..Omega_4 as printed."""
    import oracle as O
    path = os.path.join(os.path.dirname(__file__), "golden", "omega_p15.txt")
    expect = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            expect.append([int(v) for v in line.split(":")[1].split()])
    assert O.omega_levels(15) == expect


@pytest.mark.parametrize("p", [1, 2, 3, 7, 8, 15, 16, 31, 100])
def test_omega_levels_partition(p):
    import oracle as O
    levels = O.omega_levels(p)
    flat = [j for lev in levels for j in lev]
    assert sorted(flat) == list(range(1, p + 1))
    assert len(levels) == int(np.floor(np.log2(p))) + 1


# --------------------------------------------------------------------------
# accuracy properties used by the tolerances
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,s", [(1024, None), (4096, 5.88e-7)])
def test_backward_error_of_sweep(oracle, n, s):
    rng = np.random.default_rng(8)
    if s is None:
        a, b = _dominant(rng, n)
    else:
        a, b = -np.ones(n - 1), np.full(n, 2.0 + s)
    F = rng.standard_normal((n, 16))
    X = oracle.thomas_f64(a, b, F)
    R = oracle.matvec_ld(a, b, X) - F
    normA = np.max(np.abs(b) + np.r_[np.abs(a), 0] + np.r_[0, np.abs(a)])
    eta = np.abs(R).max(0) / (normA * np.abs(X).max(0) + np.abs(F).max(0))
    assert eta.max() <= 1e-14


def test_refinement_converges(oracle):
    """Three and six refinement steps agree to the limit of binary64."""
    n, s = 16384, 1e-6
    rng = np.random.default_rng(9)
    a, b = -np.ones(n - 1), np.full(n, 2.0 + s)
    F = rng.standard_normal((n, 4)).astype(np.float32).astype(np.float64)
    x3 = oracle.solve_hi(a, b, F, steps=3)
    x6 = oracle.solve_hi(a, b, F, steps=6)
    assert _rel(x3, x6) <= 4 * U64
    x0 = oracle.thomas_f64(a, b, F)
    assert _rel(x0, x6) > 1e-13        # the plain sweep is visibly worse here


# --------------------------------------------------------------------------
# gradient oracle vs central finite differences
# --------------------------------------------------------------------------

def test_grad_matches_central_differences(oracle):
    rng = np.random.default_rng(10)
    n, N = 64, 16
    a, b = rng.uniform(-1, -0.5, n - 1), rng.uniform(2.2, 3.0, n)
    F, W = rng.standard_normal((n, N)), rng.standard_normal((n, N))
    dF, da, db = oracle.grad_ld(a, b, F, W)

    def L(a_, b_, F_):
        return float(np.sum(W * oracle.solve_hi(a_, b_, F_)))

    h = 1e-6
    for i in (0, 17, 40, n - 1):
        e = np.zeros(n)
        e[i] = h
        fd = (L(a, b + e, F) - L(a, b - e, F)) / (2 * h)
        assert abs(fd - db[i]) <= 1e-6 * max(1.0, abs(db[i]))
    for i in (0, 23, n - 2):
        e = np.zeros(n - 1)
        e[i] = h
        fd = (L(a + e, b, F) - L(a - e, b, F)) / (2 * h)
        assert abs(fd - da[i]) <= 1e-6 * max(1.0, abs(da[i]))
    for (i, r) in ((0, 0), (31, 5), (n - 1, N - 1)):
        E = np.zeros((n, N))
        E[i, r] = h
        fd = (L(a, b, F + E) - L(a, b, F - E)) / (2 * h)
        assert abs(fd - dF[i, r]) <= 1e-6 * max(1.0, abs(dF[i, r]))


# --------------------------------------------------------------------------
# planted mistakes: each pin must notice a plausible oracle error
# --------------------------------------------------------------------------

def test_planted_mistakes_are_caught(oracle):
    n, s = 64, 1e-3
    ks = [1, 5, 30]
    F, X, _ = oracle.eigen_closed_form(n, 2.0 + s, ks)
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + s)
    assert _rel(oracle.solve_hi(a, b, F), X) <= 1e-12
    # sign of the off-diagonal flipped
    assert _rel(oracle.solve_hi(-a, b, F), X) > 1e-3
    # off-diagonal term dropped
    assert _rel(oracle.solve_hi(0 * a, b, F), X) > 1e-3
    # diagonal index shifted by one row
    rng = np.random.default_rng(12)
    a2, b2 = _dominant(rng, n)
    F2 = rng.standard_normal((n, 2))
    ref = oracle.gauss_ld(oracle.dense(a2, b2), F2)
    assert _rel(oracle.thomas_f64(a2, np.roll(b2, 1), F2), ref) > 1e-3
    # right-hand side rows transposed
    assert _rel(oracle.thomas_f64(a2, b2, F2[::-1]), ref) > 1e-3


# ---- nonsymmetric matrices (Section 3.5) ---------------------------------------

def _general(n, seed, eps=0.3):
    rng = np.random.default_rng(seed)
    sub = -1.0 - eps * rng.random(n - 1)
    sup = -1.0 + eps * rng.random(n - 1)
    diag = 2.5 + rng.random(n)
    return sub, diag, sup


def _dense_general(sub, diag, sup):
    return np.diag(diag) + np.diag(sub, -1) + np.diag(sup, 1)


@pytest.mark.parametrize("n", [2, 7, 40])
def test_thomas_general_matches_dense_solve(oracle, n):
    sub, diag, sup = _general(n, n)
    F = np.random.default_rng(1).standard_normal((n, 3))
    ref = np.linalg.solve(_dense_general(sub, diag, sup), F)
    assert np.max(np.abs(oracle.thomas_general(sub, diag, sup, F) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_thomas_general_matches_scipy_banded(oracle):
    linalg = pytest.importorskip("scipy.linalg")
    n = 300
    sub, diag, sup = _general(n, 9)
    F = np.random.default_rng(2).standard_normal((n, 4))
    ab = np.zeros((3, n))
    ab[0, 1:], ab[1], ab[2, :-1] = sup, diag, sub
    ref = linalg.solve_banded((1, 1), ab, F)
    assert np.max(np.abs(oracle.thomas_general(sub, diag, sup, F) - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the symmetric special case is the symmetric sweep
    a = -np.ones(n - 1)
    assert np.allclose(oracle.thomas_general(a, diag, a, F), oracle.thomas_f64(a, diag, F), rtol=0, atol=1e-14)


def test_symmetrizer_section_3_5(oracle):
    n = 25
    sub, diag, sup = _general(n, 4, eps=0.6)
    t = oracle.symmetrizer(sub, sup)
    A = _dense_general(sub, diag, sup)
    S = np.diag(1.0 / t) @ A @ np.diag(t)
    assert np.max(np.abs(S - S.T)) <= 1e-14 * np.max(np.abs(S))
    assert np.allclose(np.diag(S), diag)
    # a planted mistake (the inverse ratio) breaks the symmetry
    t_bad = 1.0 / t
    S_bad = np.diag(1.0 / t_bad) @ A @ np.diag(t_bad)
    assert np.max(np.abs(S_bad - S_bad.T)) > 1e-3


def test_algorithm2_components_equal_the_full_solve(oracle):
    """Algorithm 2 (X_k = G_k^T F, A G_k = e_k) gives the same components as the
    full solve; with every k it is the explicit inverse applied to F."""
    n, N = 300, 7
    rng = np.random.default_rng(21)
    a = -0.5 - 0.5 * rng.random(n - 1)
    b = 2.5 + rng.random(n)
    F = rng.standard_normal((n, N))
    ks = [0, 1, 57, 150, n - 2, n - 1]
    ref = oracle.solve_hi(a, b, F)[ks]
    got = oracle.algorithm2(a, b, F, ks)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    full = oracle.algorithm2(a[:39], b[:40], F[:40], np.arange(40))
    dense = np.linalg.solve(oracle.dense(a[:39], b[:40]), F[:40])
    assert np.max(np.abs(full - dense)) <= 1e-13 * np.max(np.abs(dense))
