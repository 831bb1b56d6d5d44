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


@pytest.mark.parametrize("in_dt,out_dt", [(torch.float64, torch.float64), (torch.float64, torch.float32),
                                          (torch.float32, torch.float32)])
@pytest.mark.parametrize("na,nb,S,transposed", [(33, 33, 1, False), (33, 33, 1, True), (40, 17, 37, False),
                                                (29, 29, 37, True), (64, 64, 100, True)])
def test_rhs_kernel_matches_the_difference(in_dt, out_dt, na, nb, S, transposed):
    # the half step's right-hand side h^2 (omega v + Lambda_b v + f) written out in
    # binary64 against tdm_adi_rhs, into a padded row pitch; transposed views as the
    # second half step passes them.  Binary64 inputs carry zeros and values outside
    # the binary32 pairs' range, which those elements take through binary64.
    import ctypes
    from paper_0901_2859_gb300 import _lib
    from paper_0901_2859_gb300.api import _stream_ptr, check
    g = torch.Generator().manual_seed(na * 1000 + nb * 10 + S)
    shape = (nb, na, S) if transposed else (na, nb, S)
    v = torch.randn(shape, generator=g, dtype=torch.float64)
    f = torch.randn(shape, generator=g, dtype=torch.float64)
    if in_dt == torch.float64:
        for x, seed in ((v, 1), (f, 2)):
            pick = torch.rand(shape, generator=g) < 0.05
            special = torch.tensor([0.0, 1e-30, -3e-23, 2e-22, 1e30, -1e-3], dtype=torch.float64)
            x[pick] = special[torch.randint(0, len(special), (int(pick.sum()),), generator=g)]
    v, f = v.to(in_dt).cuda(), f.to(in_dt).cuda()
    if transposed:
        v, f = v.transpose(0, 1), f.transpose(0, 1)
    h2, om = 1.0 / 1000 ** 2, 3.7e4
    c = om * h2 - 2.0
    ldR = nb * S + 5
    R = torch.full((na, ldR), 7.0, dtype=out_dt, device="cuda")
    st = _lib.load().tdm_adi_rhs(
        ctypes.c_void_p(v.data_ptr()), v.stride(0), v.stride(1), ctypes.c_void_p(f.data_ptr()), f.stride(0),
        f.stride(1), na, nb, S, c, h2, int(in_dt == torch.float64), ctypes.c_void_p(R.data_ptr()), ldR,
        int(out_dt == torch.float64), _stream_ptr(R.device))
    check(st, "tdm_adi_rhs")
    torch.cuda.synchronize()
    vd, fd = v.double().cpu(), f.double().cpu()
    ref = c * vd + h2 * fd
    ref[:, 1:] += vd[:, :-1]
    ref[:, :-1] += vd[:, 1:]
    terms = abs(c) * vd.abs() + h2 * fd.abs()          # the sum's terms' magnitudes, the error scale
    terms[:, 1:] += vd[:, :-1].abs()
    terms[:, :-1] += vd[:, 1:].abs()
    got = R.cpu()
    assert torch.all(got[:, nb * S:] == 7.0)          # the pitch's padding is left alone
    got = got[:, :nb * S].double().view(na, nb, S)
    if out_dt == torch.float64:      # binary64 sums in another order
        bound = 4 * 2.0 ** -53 * terms
    elif in_dt == torch.float64:     # within a binary32 ulp of the sum, formed in binary32 pairs (2^-47 each)
        bound = 2.0 ** -23 * ref.abs() + 2.0 ** -44 * terms
    else:                            # binary32 sums
        bound = 6 * 2.0 ** -24 * terms
    assert bool(torch.all((got - ref).abs() <= bound))
