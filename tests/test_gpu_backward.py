"""GPU gradients of L = sum(W * X), X = A^{-1} F, against the oracle's gradients.

The adjoint system is a solve with the same plan (A = A^T, Lemma 2); the
oracle's gradient is itself pinned against central finite differences in
test_oracle_pins.py.  Gates: binary64 path 1e-11, binary32 path 2e-5 relative
(max-norm over the whole vector, per quantity).
"""
import numpy as np
import pytest
import torch

from helpers import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdm():
    import paper_0901_2859_gb300 as m
    return m


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    return torch.device("cuda", 0)


def _vec_rel(x, ref):
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("n,N", [(1, 3), (2, 5), (33, 7), (1000, 37), (2049, 64)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_matches_oracle(tdm, dev, oracle, n, N, precision):
    from paper_0901_2859_gb300 import workloads
    s = workloads.diff(seed=n, n=n, N=N)
    dt = np.float64 if precision == "fp64" else np.float32
    F = s.F.astype(dt)
    W = s.W.astype(dt)
    tol = 1e-11 if precision == "fp64" else 2e-5
    plan = tdm.prepare(s.a, s.b, device=dev)
    Ft = torch.from_numpy(np.ascontiguousarray(F)).to(dev)
    Wt = torch.from_numpy(np.ascontiguousarray(W)).to(dev)
    X = plan.solve(Ft, precision)
    dF, da, db = plan.solve_backward(Wt, X, precision)
    torch.cuda.synchronize()
    rdF, rda, rdb = oracle.grad_ld(s.a, s.b, F.astype(np.float64), W.astype(np.float64))
    assert relerr(dF.cpu().numpy(), rdF) <= tol
    assert _vec_rel(db.cpu().numpy(), rdb) <= tol
    if n > 1:
        assert _vec_rel(da.cpu().numpy(), rda) <= tol
    plan.close()


def test_autograd_function(tdm, dev, oracle):
    """torch.autograd through TDMSolve gives the same gradients as the oracle."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.diff(seed=3, n=300, N=16)
    a = torch.tensor(s.a, device=dev, requires_grad=True)
    b = torch.tensor(s.b, device=dev, requires_grad=True)
    F = torch.tensor(s.F.astype(np.float64), device=dev, requires_grad=True)
    W = torch.tensor(s.W.astype(np.float64), device=dev)
    plan = tdm.prepare(a.detach(), b.detach(), device=dev)
    X = tdm.TDMSolve.apply(F, a, b, plan, "fp64")
    loss = (W * X).sum()
    loss.backward()
    rdF, rda, rdb = oracle.grad_ld(s.a, s.b, s.F.astype(np.float64), s.W.astype(np.float64))
    assert relerr(F.grad.cpu().numpy(), rdF) <= 1e-11
    assert _vec_rel(a.grad.cpu().numpy(), rda) <= 1e-11
    assert _vec_rel(b.grad.cpu().numpy(), rdb) <= 1e-11
    plan.close()


def test_backward_diff_workload_full_size(tdm, dev, oracle):
    """n = 8192, N = 2048 (the differentiation workload), binary32.

    The matrix is strongly diagonally dominant (kappa <= 25), so the oracle's
    binary64 sweep is exact to ~1e-15 and serves as the adjoint solver; the
    row sums are formed here from it in binary64 (steps=0 of the refinement).
    """
    from paper_0901_2859_gb300 import workloads
    s = workloads.diff(seed=0)
    plan = tdm.prepare(s.a, s.b, device=dev)
    Ft = torch.from_numpy(s.F).to(dev)
    Wt = torch.from_numpy(s.W).to(dev)
    X = plan.solve(Ft, "fp32")
    dF, da, db = plan.solve_backward(Wt, X, "fp32")
    torch.cuda.synchronize()
    rdF, rda, rdb = oracle.grad_ld(s.a, s.b, s.F.astype(np.float64), s.W.astype(np.float64), steps=0)
    assert relerr(dF.cpu().numpy(), rdF) <= 2e-5
    assert _vec_rel(db.cpu().numpy(), rdb) <= 2e-5
    assert _vec_rel(da.cpu().numpy(), rda) <= 2e-5
    plan.close()


def test_backward_is_deterministic(tdm, dev):
    from paper_0901_2859_gb300 import workloads
    s = workloads.diff(seed=5, n=4000, N=300)
    plan = tdm.prepare(s.a, s.b, device=dev)
    Ft = torch.from_numpy(s.F).to(dev)
    Wt = torch.from_numpy(s.W).to(dev)
    X = plan.solve(Ft, "fp32")
    r1 = plan.solve_backward(Wt, X, "fp32")
    r2 = plan.solve_backward(Wt, X, "fp32")
    torch.cuda.synchronize()
    for u, v in zip(r1, r2):
        assert torch.equal(u, v)
    plan.close()


def test_refined_backward_ill_conditioned(tdm, dev, oracle):
    """TDM_FP32_REFINED backward: Lambda = A^{-1} W by the refined solve (W
    binary32, Lambda binary64), the row sums in binary64.  a = -1, b = 2 + 1e-6,
    n = 4096 (kappa ~ 2.5e6): dF, da and db within 1e-11 of the oracle's
    long-double gradient."""
    n, N = 4096, 16
    rng = np.random.default_rng(41)
    a, b = -np.ones(n - 1), np.full(n, 2.0 + 1e-6)
    F = rng.standard_normal((n, N)).astype(np.float32)
    W = rng.standard_normal((n, N)).astype(np.float32)
    plan = tdm.prepare(a, b, device=dev)
    X = plan.solve(torch.from_numpy(F).to(dev), "fp32_refined")
    dF, da, db = plan.solve_backward(torch.from_numpy(W).to(dev), X, "fp32_refined")
    torch.cuda.synchronize()
    assert dF.dtype == torch.float64
    rdF, rda, rdb = oracle.grad_ld(a, b, F.astype(np.float64), W.astype(np.float64))
    assert relerr(dF.cpu().numpy(), rdF) <= 1e-11
    assert _vec_rel(db.cpu().numpy(), rdb) <= 1e-11
    assert _vec_rel(da.cpu().numpy(), rda) <= 1e-11
    assert plan.info()["device_error"] == 0
    plan.close()


def test_autograd_refined(tdm, dev, oracle):
    """torch.autograd through TDMSolve with the refined precision: F binary32
    (its gradient too), a and b binary64."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.diff(seed=7, n=500, N=12)
    a = torch.tensor(s.a, device=dev, requires_grad=True)
    b = torch.tensor(s.b, device=dev, requires_grad=True)
    F = torch.tensor(s.F, device=dev, requires_grad=True)             # binary32
    W = torch.tensor(s.W.astype(np.float64), device=dev)              # binary32 values
    plan = tdm.prepare(a.detach(), b.detach(), device=dev)
    X = tdm.TDMSolve.apply(F, a, b, plan, "fp32_refined")
    assert X.dtype == torch.float64
    (W * X).sum().backward()
    rdF, rda, rdb = oracle.grad_ld(s.a, s.b, s.F.astype(np.float64), s.W.astype(np.float64))
    assert F.grad.dtype == torch.float32
    assert relerr(F.grad.double().cpu().numpy(), rdF) <= 2 ** -23
    assert _vec_rel(a.grad.cpu().numpy(), rda) <= 1e-11
    assert _vec_rel(b.grad.cpu().numpy(), rdb) <= 1e-11
    plan.close()


def test_gradient_against_central_differences_on_a_subblock(tdm, dev, oracle):
    """The differentiation workload at full size (n = 8192, N = 2048): the GPU
    gradient of L = sum(W * X) against binary64 central differences with step
    1e-6, on a 64 x 16 sub-block of F (each difference moves one column of X:
    L's change is that column's) and on 16 entries each of a and b (every column
    moves).  The differences themselves are accurate to ~1e-6 (rounding / step),
    which sets the gate; the tight check is the oracle gradient above."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.diff(seed=0)
    n, N, h = s.n, s.N, 1e-6
    rows, cols = np.arange(3000, 3064), np.arange(100, 116)
    F64, W64 = s.F.astype(np.float64), s.W.astype(np.float64)
    plan = tdm.prepare(s.a, s.b, device=dev)
    Ft, Wt = torch.from_numpy(s.F).to(dev), torch.from_numpy(s.W).to(dev)
    grads = {}
    for prec in ("fp32_refined", "fp32"):
        X = plan.solve(Ft, prec)
        grads[prec] = [g.cpu().numpy() if g is not None else None for g in plan.solve_backward(Wt, X, prec)]
    torch.cuda.synchronize()
    # dL/dF on the sub-block: one column's solve per difference
    fd = np.empty((len(rows), len(cols)))
    for jj, j in enumerate(cols):
        Fp = np.repeat(F64[:, j:j + 1], 2 * len(rows), axis=1)
        for ii, i in enumerate(rows):
            Fp[i, 2 * ii] += h
            Fp[i, 2 * ii + 1] -= h
        Xp = oracle.thomas_f64(s.a, s.b, Fp)
        Lp = W64[:, j] @ Xp
        fd[:, jj] = (Lp[0::2] - Lp[1::2]) / (2 * h)
    # dL/db and dL/da on 16 rows: every column moves
    ab_rows = rows[::4]
    fdb, fda = np.empty(len(ab_rows)), np.empty(len(ab_rows))
    for k, i in enumerate(ab_rows):
        for which, out in (("b", fdb), ("a", fda)):
            Ls = []
            for sgn in (1.0, -1.0):
                a2, b2 = s.a.copy(), s.b.copy()
                (b2 if which == "b" else a2)[i] += sgn * h
                Ls.append(float(np.sum(W64 * oracle.thomas_f64(a2, b2, F64))))
            out[k] = (Ls[0] - Ls[1]) / (2 * h)
    for prec, (dF, da, db) in grads.items():
        assert relerr(dF[np.ix_(rows, cols)], fd) <= 1e-5, prec
        assert _vec_rel(db[ab_rows], fdb) <= 1e-5, prec
        assert _vec_rel(da[ab_rows], fda) <= 1e-5, prec
    plan.close()
