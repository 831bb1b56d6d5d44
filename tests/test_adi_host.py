"""Host logic of the alternating-direction solver (Section 4b) on CPU: the
half steps' layouts, transposes and precisions, with the library's solve
replaced by the oracle's sweep (a fake plan) and its right-hand-side kernel by
the three-point difference written out here, against the oracle's iteration;
and the parameters against the oracle's.  The kernel itself is compared with
that difference on the GPU."""
import numpy as np
import pytest
import torch


class _FakePlan:
    def __init__(self, a, b):
        self.a, self.b = a, b

    def solve(self, F, precision, out):
        import oracle
        out.copy_(torch.from_numpy(oracle.thomas_f64(self.a, self.b, F.double().numpy())).to(out.dtype))
        return out


def _fake_rhs(pr):
    """The half step's right-hand side h^2 (omega v + Lambda_b v + f), u = 0 beyond
    the ends of b, into buf[a, (b, s)] in buf's precision."""
    def rhs(v, f, om, buf):
        n, _, S = v.shape
        h2 = 1.0 / (pr.N * pr.N)
        r = v.double().clone() * (om * h2 - 2.0) + h2 * f.double()
        r[:, 1:] += v[:, :-1].double()
        r[:, :-1] += v[:, 1:].double()
        buf[:, :n * S].view(n, n, S).copy_(r)
    return rhs


def _fake_solver(N, eps, precision):
    from paper_0901_2859_gb300.adi import PeacemanRachford, adi_parameters
    pr = PeacemanRachford.__new__(PeacemanRachford)
    pr.N, pr.eps, pr.precision, pr.device = N, eps, precision, torch.device("cpu")
    pr.omegas = adi_parameters(N, eps)
    n, h = N - 1, 1.0 / N
    pr.plans = [_FakePlan(-np.ones(n - 1), np.full(n, 2.0 + om * h * h)) for om in pr.omegas]
    pr._rhs = _fake_rhs(pr)
    return pr


def test_parameters_match_the_oracle():
    from oracle import poisson as op
    from paper_0901_2859_gb300.adi import adi_parameters
    for N, eps in ((64, 1e-3), (1024, 1e-5), (2, 0.5)):
        assert np.allclose(adi_parameters(N, eps), op.adi_parameters(N, eps), rtol=1e-14, atol=0)
    with pytest.raises(ValueError):
        adi_parameters(1, 1e-5)


@pytest.mark.parametrize("S,precision", [(1, "fp64"), (3, "fp64"), (2, "fp32_refined")])
def test_iteration_matches_the_oracle(S, precision):
    from oracle import poisson as op
    N = 20
    pr = _fake_solver(N, 1e-4, precision)
    f = np.random.default_rng(S).standard_normal((N - 1, N - 1, S))
    got = pr.solve(torch.from_numpy(f)).numpy()
    ref = op.peaceman_rachford(f, N, op.adi_parameters(N, 1e-4))
    # fp32_refined rounds each right-hand side to binary32 (the fake plan then solves it exactly)
    assert np.max(np.abs(got - ref)) <= (1e-12 if precision == "fp64" else 1e-6) * np.max(np.abs(ref))
    got2 = pr.solve(torch.from_numpy(f[:, :, 0])).numpy()
    assert got2.shape == (N - 1, N - 1) and np.allclose(got2, got[:, :, 0], rtol=0, atol=1e-13)
