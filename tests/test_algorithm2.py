"""Algorithm 2 (Section 3.1): selected components as G_k^T F.  On CPU: the TF32
split is exact.  On the GPU: the tensor-core kernel (three TF32 products,
binary32 accumulation over at most 1024 rows of K) and the binary64 product
against the oracle's Algorithm 2 and the full solve, on ragged shapes and on
the ill-conditioned precision series."""
import numpy as np
import pytest
import torch

from helpers import relerr

TOL_TC = 2e-5    # the binary32 gate
TOL_64 = 1e-11


def test_tf32_split_is_exact():
    from paper_0901_2859_gb300.algorithm2 import _tf32_split
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(10000).astype(np.float32))
    head, tail = _tf32_split(x)
    assert torch.equal(head + tail, x)
    assert int((head.view(torch.int32) & 0x1FFF).abs().max()) == 0   # 10 significand bits kept
    assert float((tail.abs() / x.abs().clamp_min(1e-30)).max()) < 2.0 ** -10


@pytest.mark.gpu
@pytest.mark.parametrize("mode,tol", [("fp64", TOL_64), ("tc", TOL_TC)])
def test_components_match_oracle_and_full_solve(oracle, mode, tol):
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    from paper_0901_2859_gb300.algorithm2 import components, inverse_rows
    s = workloads.random_dominant(seed=31, n=3000, N=50)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    ks = [0, 1, 999, 1000, 2047, 2999]
    F = torch.from_numpy(s.F.astype(np.float32)).cuda()
    X = components(plan, F, ks, mode).double().cpu().numpy()
    F64 = s.F.astype(np.float32).astype(np.float64)
    ref = oracle.algorithm2(s.a, s.b, F64, ks)
    assert relerr(X.T, ref.T) <= tol
    full = plan.solve(F.double(), "fp64").cpu().numpy()[ks]
    assert relerr(X.T, full.T) <= tol
    G = inverse_rows(plan, ks)          # reused across calls
    assert torch.equal(components(plan, F, ks, mode, G=G), components(plan, F, ks, mode, G=G))
    with pytest.raises(ValueError):
        inverse_rows(plan, [3000])
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n,N,P", [(100, 1, 1), (1000, 5, 37), (3000, 130, 511), (2100, 300, 600)])
def test_tensor_core_product_on_ragged_shapes(n, N, P):
    """n not a multiple of the 16-row stage or the 1024-row slice, N not a
    multiple of 4 or of the 128-column tile, P across the 512-component block:
    the kernel against the binary64 product of the same G and F."""
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    from paper_0901_2859_gb300.algorithm2 import components, inverse_rows
    s = workloads.random_dominant(seed=n + N, n=n, N=N)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    rng = np.random.default_rng(P)
    ks = np.sort(rng.choice(n, size=min(P, n), replace=P > n))
    F = torch.from_numpy(s.F.astype(np.float32)).cuda()
    G = inverse_rows(plan, ks)
    X = components(plan, F, ks, "tc", G=G).double().cpu().numpy()
    ref = components(plan, F, ks, "fp64", G=G).cpu().numpy()
    assert X.shape == (len(ks), N)
    assert relerr(X.T, ref.T) <= TOL_TC
    plan.close()


@pytest.mark.gpu
def test_tensor_core_product_on_the_precision_series(oracle):
    """n = 16384, a = -1, b = 2 + 1e-6 (kappa ~ 4e6), every separator of the
    plan (511 components): G_k^T F cancels heavily (|x_k| << sum |G_k(i) F_i|),
    which one binary32 accumulation over all 16384 rows does not survive; the
    kernel's slices of 1024 rows, added in binary32 pairs, stay within 2e-5 of
    the oracle's solution."""
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    from paper_0901_2859_gb300.algorithm2 import components, inverse_rows
    s = workloads.precision(seed=0, n=16384, N=256, s=1e-6)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    t = plan.info()["block_rows"]
    ks = list(range(t, s.n, t))
    F = torch.from_numpy(s.F).cuda()
    G = inverse_rows(plan, ks)
    X = components(plan, F, ks, "tc", G=G).double().cpu().numpy()
    cols = np.r_[0:8, 120:128, 248:256]
    ref = oracle.solve_hi(s.a, s.b, np.ascontiguousarray(s.F[:, cols], dtype=np.float64))[ks]
    assert relerr(X[:, cols].T, ref.T) <= TOL_TC
    plan.close()
