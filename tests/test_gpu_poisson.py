"""The Fourier Poisson solver (Section 4a) on the GPU against the oracle: the
model problem's discrete solution in closed form, random series, both
precisions, and the type-I sine transform against the explicit sine sums."""
import numpy as np
import pytest
import torch

from helpers import relerr

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    """max |x - ref| / max |ref| over the whole mesh (the model solution has zero lines)"""
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    return torch.device("cuda", 0)


def test_dst1_matches_sine_sums(dev):
    from oracle import poisson as op
    from paper_0901_2859_gb300.poisson import dst1
    x = np.random.default_rng(0).standard_normal((5, 37, 3))
    got = dst1(torch.from_numpy(x).to(dev), dim=1).cpu().numpy()
    ref = np.einsum("lj,ijn->iln", op.sine_matrix(38), x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("N1,N2", [(64, 64), (48, 80), (129, 33)])
def test_model_problem(dev, precision, N1, N2):
    from oracle import poisson as op
    from paper_0901_2859_gb300.poisson import FourierPoisson
    f, u, h1, h2 = op.model_problem(N1, N2)
    fp = FourierPoisson(N1, N2, precision=precision, device=dev)
    got = fp.solve(FourierPoisson.model_rhs(N1, N2, device=dev))
    torch.cuda.synchronize()
    assert _rel(got.cpu().numpy(), u) <= 1e-11
    fp.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_random_series_matches_oracle(dev, precision):
    from oracle import poisson as op
    from paper_0901_2859_gb300.poisson import FourierPoisson
    N1, N2, h1, h2 = 40, 24, 0.03, 0.05
    f = np.random.default_rng(5).standard_normal((N1 - 1, N2 - 1, 6))
    fp = FourierPoisson(N1, N2, h1, h2, precision=precision, device=dev)
    got = fp.solve(torch.from_numpy(f).to(dev)).cpu().numpy()
    ref = op.fourier_poisson(f, h1, h2)
    assert relerr(got, ref) <= 1e-11
    assert np.max(np.abs(op.laplacian(got, h1, h2) + f)) <= 1e-8 * np.max(np.abs(f))
    fp.close()


def test_unsplit_binary32_rhs_is_binary32_accurate(dev):
    from oracle import poisson as op
    from paper_0901_2859_gb300.poisson import FourierPoisson
    N1, N2 = 50, 30
    f = np.random.default_rng(9).standard_normal((N1 - 1, N2 - 1, 2))
    fp = FourierPoisson(N1, N2, device=dev, rhs_split=False)
    err = relerr(fp.solve(torch.from_numpy(f).to(dev)).cpu().numpy(), op.fourier_poisson(f, 1 / N1, 1 / N2))
    assert 1e-12 < err <= 1e-6   # the binary32 rounding of the coefficients, not the solves
    fp.close()


def test_bad_shapes_rejected(dev):
    from paper_0901_2859_gb300.poisson import FourierPoisson
    fp = FourierPoisson(8, 8, device=dev)
    with pytest.raises(ValueError):
        fp.solve(torch.zeros(6, 7, device=dev, dtype=torch.float64))
    with pytest.raises(ValueError):
        FourierPoisson(1, 8, device=dev)
    fp.close()
