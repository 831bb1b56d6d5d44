"""Algorithm 2 (Section 3.1): selected components as G_k^T F.  On CPU: the TF32
split is exact.  On the GPU: both products against the oracle's Algorithm 2 and
the full solve."""
import numpy as np
import pytest
import torch

from helpers import relerr


def test_tf32_split_is_exact():
    from paper_0901_2859_gb300.algorithm2 import _tf32_split
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(10000).astype(np.float32))
    head, tail = _tf32_split(x)
    assert torch.equal(head + tail, x)
    assert int((head.view(torch.int32) & 0x1FFF).abs().max()) == 0   # 10 significand bits kept
    assert float((tail.abs() / x.abs().clamp_min(1e-30)).max()) < 2.0 ** -10


@pytest.mark.gpu
@pytest.mark.parametrize("mode,tol", [("fp64", 1e-11), ("tf32x3", 2e-5)])
def test_components_match_oracle_and_full_solve(oracle, mode, tol):
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    from paper_0901_2859_gb300.algorithm2 import components, inverse_rows
    s = workloads.random_dominant(seed=31, n=3000, N=50)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    ks = [0, 1, 999, 1000, 2047, 2999]
    F = torch.from_numpy(s.F).cuda()
    X = components(plan, F, ks, mode).double().cpu().numpy()
    ref = oracle.algorithm2(s.a, s.b, s.F, ks)
    assert relerr(X.T, ref.T) <= tol
    full = plan.solve(F, "fp64").cpu().numpy()[ks]
    assert relerr(X.T, full.T) <= tol
    G = inverse_rows(plan, ks)          # reused across calls
    assert torch.equal(components(plan, F, ks, mode, G=G), components(plan, F, ks, mode, G=G))
    with pytest.raises(ValueError):
        inverse_rows(plan, [3000])
    plan.close()
