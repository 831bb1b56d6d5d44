"""Failure detection without a GPU fault: a bounded device wait that nothing
completes (an mbarrier, or a group barrier whose member never arrives) gives
up and reports, and a refinement that cannot converge within its cap reports
device error 2; the context stays usable after each."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports():
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import _lib, workloads
    lib = _lib.load()
    assert lib.tdm_selftest_wait_timeout(1 << 22, None) == 6     # TDM_ERR_TIMEOUT, in a few ms
    s = workloads.plain_fp64(seed=0, n=500, N=8)                 # the context still works
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    X = plan.solve(torch.from_numpy(s.F).cuda(), "fp64")
    torch.cuda.synchronize()
    assert torch.isfinite(X).all() and plan.info()["device_error"] == 0
    plan.close()


def test_group_barrier_gives_up_and_reports():
    """The group barrier of the cooperative launches: a member that never
    arrives makes the other's bounded wait give up with device error 3
    (TDM_ERR_TIMEOUT from the self-test); the context then still solves, in
    the cooperative form too."""
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import _lib, workloads
    lib = _lib.load()
    assert lib.tdm_selftest_group_timeout(1 << 12, None) == 6
    s = workloads.precision(seed=1, n=16384, N=40, s=1e-2)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    X = plan.solve(torch.from_numpy(s.F).cuda(), "fp32_refined")
    torch.cuda.synchronize()
    assert torch.isfinite(X).all() and plan.info()["device_error"] == 0
    plan.close()


def test_refinement_cap_reports_non_convergence():
    import paper_0901_2859_gb300 as tdm
    n = 16384
    a = -np.ones(n - 1)
    # the Dirichlet Laplacian shifted to a smallest eigenvalue of 1e-10 (kappa ~ 4e10): its binary32
    # rounding moves the spectrum by more than that, so the binary32 corrections cannot converge
    # (its binary64 LU pivots all stay near 1, so prepare accepts it)
    lam1 = 2.0 - 2.0 * np.cos(np.pi / (n + 1))
    b = np.full(n, 2.0 - lam1 + 1e-10)
    plan = tdm.prepare(a, b, refine_steps=-1, device="cuda:0")
    F = torch.from_numpy(np.random.default_rng(0).standard_normal((n, 16)).astype(np.float32)).cuda()
    plan.solve(F, "fp32_refined")
    torch.cuda.synchronize()
    assert plan.info()["device_error"] == 2
    plan.close()
    good = tdm.prepare(-np.ones(99), np.full(100, 2.5), device="cuda:0")   # a new plan is unaffected
    good.solve(F[:100].contiguous(), "fp32_refined")
    torch.cuda.synchronize()
    assert good.info()["device_error"] == 0
    good.close()
