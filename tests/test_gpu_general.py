"""Nonsymmetric tridiagonal matrices (Section 3.5) on the GPU: the plan of the
symmetrized matrix with the similarity folded into its coefficients, against
the oracle's general sweep; the symmetric special case; and the combinations
that a general plan rejects."""
import numpy as np
import pytest
import torch

from helpers import relerr

pytestmark = pytest.mark.gpu


def _general(n, seed, eps):
    rng = np.random.default_rng(seed)
    sub = -1.0 - eps * rng.random(n - 1)
    sup = -1.0 + eps * rng.random(n - 1)
    diag = 2.2 + rng.random(n)
    return sub, diag, sup


@pytest.mark.parametrize("n", [1, 2, 33, 1000, 5000])
@pytest.mark.parametrize("block_rows", [16, 32])
@pytest.mark.parametrize("eps", [0.3, 0.9])
def test_matches_general_sweep(oracle, n, block_rows, eps):
    import paper_0901_2859_gb300 as tdm
    sub, diag, sup = _general(n, n + block_rows, eps)
    F = np.random.default_rng(n).standard_normal((n, 21))
    ref = oracle.thomas_general(sub, diag, sup, F)
    plan = tdm.prepare_general(sub, diag, sup, block_rows=block_rows, device="cuda:0")
    assert plan.info()["general"] == 1
    X64 = plan.solve(torch.from_numpy(F).cuda(), "fp64").cpu().numpy()
    assert relerr(X64, ref) <= 1e-12
    X32 = plan.solve(torch.from_numpy(F.astype(np.float32)).cuda(), "fp32").cpu().numpy()
    assert relerr(X32, oracle.thomas_general(sub, diag, sup, F.astype(np.float32).astype(np.float64))) <= 2e-5
    plan.close()


def test_symmetric_special_case_is_the_symmetric_plan():
    import paper_0901_2859_gb300 as tdm
    n = 3000
    rng = np.random.default_rng(5)
    a = -0.5 - 0.5 * rng.random(n - 1)
    b = 2.5 + rng.random(n)
    F = torch.from_numpy(rng.standard_normal((n, 10))).cuda()
    p1 = tdm.prepare(a, b, device="cuda:0")
    p2 = tdm.prepare_general(a, b, a, device="cuda:0")
    assert torch.equal(p1.solve(F, "fp64"), p2.solve(F, "fp64"))
    p1.close()
    p2.close()


def test_batched_general_plans(oracle):
    import paper_0901_2859_gb300 as tdm
    plans, Fs, refs = [], [], []
    for k, n in enumerate((100, 700, 2500)):
        sub, diag, sup = _general(n, 40 + k, 0.5)
        F = np.random.default_rng(k).standard_normal((n, 12))
        plans.append(tdm.prepare_general(sub, diag, sup, device="cuda:0"))
        Fs.append(torch.from_numpy(F).cuda())
        refs.append(oracle.thomas_general(sub, diag, sup, F))
    for X, ref in zip(tdm.solve_batched(plans, Fs, "fp64"), refs):
        assert relerr(X.cpu().numpy(), ref) <= 1e-12
    for p in plans:
        p.close()


def test_rejections():
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import TDMError
    n = 64
    sub, diag, sup = _general(n, 1, 0.3)
    bad = sup.copy()
    bad[10] = -bad[10]          # sub * sup < 0 at one row: no real similarity
    with pytest.raises(TDMError) as e:
        tdm.prepare_general(sub, diag, bad, device="cuda:0")
    assert e.value.status == 1
    plan = tdm.prepare_general(sub, diag, sup, device="cuda:0")
    F32 = torch.zeros((n, 4), dtype=torch.float32, device="cuda:0")
    with pytest.raises(TDMError) as e:
        plan.solve(F32, "fp32_refined")
    assert e.value.status == 7
    with pytest.raises(TDMError) as e:
        plan.solve_backward(F32, F32, "fp32")
    assert e.value.status == 7
    plan.close()
