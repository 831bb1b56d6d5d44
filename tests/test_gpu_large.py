"""Systems beyond one cluster: the two-level scheme (segments solved by their own
plans, the separator values from a reduced plan) against the oracle, in every
precision, with sampled columns; and the host-buffer path on such a plan."""
import numpy as np
import pytest
import torch

from helpers import relerr

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32_refined": 1e-11, "fp32": 2e-5}


@pytest.mark.parametrize("n", [32769, 70001, 200000])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined", "fp32"])
def test_two_level_matches_oracle(oracle, n, precision):
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    s = workloads.random_dominant(seed=n, n=n, N=9)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    F = torch.from_numpy(s.F).to("cuda:0", dt)
    X = plan.solve(F, precision).double().cpu().numpy()
    ref = oracle.solve_hi(s.a, s.b, F.double().cpu().numpy())
    assert relerr(X, ref) <= TOL[precision]
    assert plan.info()["device_error"] == 0
    plan.close()


def test_two_level_poisson_shift_and_block_rows(oracle):
    """An ill-conditioned shifted Laplacian (kappa ~ 4e6) across 3 segments of 16-row blocks."""
    import paper_0901_2859_gb300 as tdm
    n = 40000
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + 1e-6)
    F = np.random.default_rng(3).standard_normal((n, 6))
    plan = tdm.prepare(a, b, block_rows=16, device="cuda:0")
    X = plan.solve(torch.from_numpy(F).cuda(), "fp64").cpu().numpy()
    assert relerr(X, oracle.solve_hi(a, b, F)) <= 1e-10
    X32 = plan.solve(torch.from_numpy(F.astype(np.float32)).cuda(), "fp32_refined").cpu().numpy()
    assert relerr(X32, oracle.solve_hi(a, b, F.astype(np.float32).astype(np.float64))) <= 1e-11
    plan.close()


def test_two_level_host_buffers():
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    s = workloads.random_dominant(seed=5, n=50000, N=40)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    F = torch.from_numpy(s.F).float().pin_memory()
    X = plan.solve_host(F, "fp32_refined", chunk=16)
    torch.cuda.synchronize()
    assert torch.equal(X, plan.solve(F.cuda(), "fp32_refined").cpu())
    plan.close()
