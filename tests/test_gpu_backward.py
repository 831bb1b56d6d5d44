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
