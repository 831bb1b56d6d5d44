"""The alternating-direction solver (Section 4b) on the GPU: the iteration
against the oracle's, element by element, and the accuracy eps reached against
the exact discrete solution of the model problem and the Fourier solution."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32_refined", 1e-7), ("fp32", 1e-4)])
def test_iteration_matches_the_oracle(precision, tol):
    from oracle import poisson as op
    from paper_0901_2859_gb300.adi import PeacemanRachford
    N, eps = 96, 1e-4
    f = np.random.default_rng(4).standard_normal((N - 1, N - 1, 3))
    pr = PeacemanRachford(N, eps, precision=precision, device="cuda:0")
    got = pr.solve(torch.from_numpy(f).cuda()).double().cpu().numpy()
    assert _rel(got, op.peaceman_rachford(f, N, op.adi_parameters(N, eps))) <= tol
    pr.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("N", [64, 257])
def test_reaches_eps(precision, N):
    from oracle import poisson as op
    from paper_0901_2859_gb300.adi import PeacemanRachford
    eps = 1e-5
    f, u, _, _ = op.model_problem(N, N)
    pr = PeacemanRachford(N, eps, precision=precision, device="cuda:0")
    assert _rel(pr.solve(torch.from_numpy(f).cuda()).double().cpu().numpy(), u) <= eps
    fr = np.random.default_rng(N).standard_normal((N - 1, N - 1, 2))
    ref = op.fourier_poisson(fr, 1.0 / N, 1.0 / N)
    assert _rel(pr.solve(torch.from_numpy(fr).cuda()).double().cpu().numpy(), ref) <= eps
    pr.close()


@pytest.mark.parametrize("N", [64, 257])
def test_binary32_within_its_rounding(N):
    # binary32 state and solves: the iteration error plus the binary32 solves' rounding
    from oracle import poisson as op
    from paper_0901_2859_gb300.adi import PeacemanRachford
    f, u, _, _ = op.model_problem(N, N)
    pr = PeacemanRachford(N, 1e-5, precision="fp32", device="cuda:0")
    assert _rel(pr.solve(torch.from_numpy(f).cuda()).double().cpu().numpy(), u) <= 1e-4
    pr.close()


def test_bad_arguments_rejected():
    from paper_0901_2859_gb300.adi import PeacemanRachford
    with pytest.raises(ValueError):
        PeacemanRachford(16, precision="bf16", device="cuda:0")
    pr = PeacemanRachford(16, device="cuda:0")
    with pytest.raises(ValueError):
        pr.solve(torch.zeros(15, 14, device="cuda:0"))
    pr.close()
