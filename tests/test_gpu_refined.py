"""GPU parity of the refined path (binary32 solves + error-free residuals,
binary64 output) against the oracle's long-double-refined solve.

Gate: relative max-norm error <= 1e-11 per column against the oracle solve of
the same binary32 right-hand sides (the refined path's target accuracy)."""
import numpy as np
import pytest
import torch

from helpers import U64, relerr

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def tdm():
    import paper_0901_2859_gb300 as m
    return m


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    return torch.device("cuda", 0)


def _refined(tdm, dev, a, b, F32, block_rows=0, steps=0):
    plan = tdm.prepare(a, b, block_rows=block_rows, refine_steps=steps, device=dev)
    X = plan.solve(torch.from_numpy(np.ascontiguousarray(F32)).to(dev), "fp32_refined")
    torch.cuda.synchronize()
    out = X.cpu().numpy()
    info = plan.info()
    plan.close()
    assert info["device_error"] == 0
    return out


@pytest.mark.parametrize("block_rows", [16, 32])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 64, 65, 100, 1023, 1025, 4097])
def test_refined_edge_sizes(tdm, dev, oracle, n, block_rows):
    from paper_0901_2859_gb300 import workloads
    s = workloads.random_dominant(seed=n + 7, n=n, N=33)
    F32 = s.F.astype(np.float32)
    ref = oracle.solve_hi(s.a, s.b, F32.astype(np.float64))
    assert relerr(_refined(tdm, dev, s.a, s.b, F32, block_rows), ref) <= TOL


@pytest.mark.parametrize("N", [1, 5, 16, 17, 40, 64])
def test_refined_ragged_rhs_counts_and_alignment(tdm, dev, oracle, N):
    """Column counts below, at and between multiples of the tile width (ragged last tiles)."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.plain_fp64(seed=N, n=2000, N=N)
    F32 = s.F.astype(np.float32)
    ref = oracle.solve_hi(s.a, s.b, F32.astype(np.float64))
    assert relerr(_refined(tdm, dev, s.a, s.b, F32), ref) <= TOL


@pytest.mark.parametrize("s_shift", [1e-6, 1e-4, 1e-2, 1.0])
def test_refined_precision_workload_sampled(tdm, dev, oracle, s_shift):
    """Full size n = 16384, N = 8192 (the benchmark's launch); sampled columns."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.precision(seed=2, s=s_shift)
    plan = tdm.prepare(s.a, s.b, device=dev)
    X = plan.solve(torch.from_numpy(s.F).to(dev), "fp32_refined")
    torch.cuda.synchronize()
    cols = np.r_[0:3, 16:19, 4095:4098, s.N - 3:s.N]
    Xc = X[:, cols].cpu().numpy()
    ref = oracle.solve_hi(s.a, s.b, np.ascontiguousarray(s.F[:, cols], dtype=np.float64))
    err = relerr(Xc, ref)
    assert err <= TOL, err
    assert plan.info()["device_error"] == 0
    plan.close()


U_PAIR = 2.0 ** -48   # unit roundoff of the binary32-pair arithmetic of the residual


def residual_floor(lam_k, lam_min):
    """Accuracy floor of the refined path for a pure sine mode k.

    The residual of a mode-k iterate is formed from fluxes of size
    sqrt(lam_k) |x| with a pair rounding error ~U_PAIR of that; the correction
    solve maps this noise into the smooth modes, amplified by 1/lam_min.  With
    the projection of random noise on the smooth modes (~0.1 measured bound):
    floor = 0.1 * U_PAIR * sqrt(lam_k) / lam_min.  For k ~ n at kappa ~ 3.4e6
    this is ~1e-10; for mixed right-hand sides |x| is dominated by the smooth
    modes and the floor is far below 1e-11.
    """
    return 0.1 * U_PAIR * np.sqrt(lam_k) / lam_min


def test_refined_poisson2d_pure_and_mixed_modes(tdm, dev, oracle):
    """n = N = 4096, kappa ~ 3.4e6: pure sine modes (closed form) and mode + noise columns."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.poisson2d(seed=1)
    n = s.n
    ks = [1, 2, 3, n // 2, n - 1, n]
    Fe, Xe, lam = oracle.eigen_closed_form(n, s.b[0], ks)
    Fe32 = Fe.astype(np.float32)
    Xr = _refined(tdm, dev, s.a, s.b, Fe32)
    ref = oracle.solve_hi(s.a, s.b, Fe32.astype(np.float64))
    errs = [relerr(Xr[:, c], ref[:, c]) for c in range(len(ks))]
    tols = [max(TOL, residual_floor(lam[c], lam.min())) for c in range(len(ks))]
    assert all(e <= t for e, t in zip(errs, tols)), list(zip(ks, errs, tols))
    assert all(e <= TOL for e, k in zip(errs, ks) if k <= 3), list(zip(ks, errs))   # smooth modes
    cols = np.r_[64:80]
    F32 = np.ascontiguousarray(s.F[:, cols], dtype=np.float32)
    ref = oracle.solve_hi(s.a, s.b, F32.astype(np.float64))
    assert relerr(_refined(tdm, dev, s.a, s.b, F32), ref) <= TOL


def test_refined_beats_plain_binary64_accuracy_when_ill_conditioned(tdm, dev, oracle):
    """At s = 1e-6 the refined result is closer to the truth than a binary64 solve can be."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.precision(seed=3, n=16384, N=16, s=1e-6)
    ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
    e_ref = relerr(_refined(tdm, dev, s.a, s.b, s.F), ref)
    e_sweep = relerr(oracle.thomas_f64(s.a, s.b, s.F.astype(np.float64)), ref)
    assert e_ref <= TOL and e_ref < e_sweep


@pytest.mark.parametrize("steps", [-1, 1, 2, 3, 4])
def test_refinement_step_counts(tdm, dev, oracle, steps):
    """A well-conditioned matrix reaches the gate with any step count >= 1."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.plain_fp64(seed=9, n=1024, N=32)
    F32 = s.F.astype(np.float32)
    ref = oracle.solve_hi(s.a, s.b, F32.astype(np.float64))
    assert relerr(_refined(tdm, dev, s.a, s.b, F32, steps=steps), ref) <= TOL


def test_automatic_refinement_is_calibrated_per_plan(tdm, dev, oracle):
    """refine_steps = 0: prepare measures the contraction of one correction on
    seeded right-hand sides, and every tile tests its first correction against
    it.  The first solve keeps x as a binary32 pair, so on the precision
    workload's worst case (s = 1e-6, kappa ~ 3.9e6) every tile of N(0,1)
    columns stops after one correction: the result equals the one-correction
    solve bit for bit.  Requested explicitly, -1 keeps contraction 1 (at least
    two corrections); both meet the gate."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.precision(seed=0, n=16384, N=64, s=1e-6)
    auto = tdm.prepare(s.a, s.b, device=dev)
    info = auto.info()
    assert info["refine_steps"] == -1
    assert 0.0 < info["contraction"] < 1e-4
    one = tdm.prepare(s.a, s.b, refine_steps=1, device=dev)
    tested = tdm.prepare(s.a, s.b, refine_steps=-1, device=dev)
    assert tested.info()["refine_steps"] == -1 and tested.info()["contraction"] == 1.0
    F = torch.from_numpy(s.F).to(dev)
    Xa = auto.solve(F, "fp32_refined")
    X1 = one.solve(F, "fp32_refined")
    Xt = tested.solve(F, "fp32_refined")
    torch.cuda.synchronize()
    assert torch.equal(Xa, X1)
    ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
    assert relerr(Xa.cpu().numpy(), ref) <= TOL
    assert relerr(Xt.cpu().numpy(), ref) <= TOL
    for q in (auto, one, tested):
        assert q.info()["device_error"] == 0
    well = workloads.plain_fp64(seed=4, n=1000, N=8)
    p = tdm.prepare(well.a, well.b, device=dev)
    assert p.info()["refine_steps"] == -1 and p.info()["contraction"] < 1e-4
    for q in (auto, one, tested, p):
        q.close()


def test_largest_refined_size_and_the_next(tdm, dev, oracle):
    from paper_0901_2859_gb300 import workloads
    n = 65536
    s = workloads.random_dominant(seed=9, n=n, N=12)
    F32 = s.F.astype(np.float32)
    ref = oracle.solve_hi(s.a, s.b, F32.astype(np.float64))
    assert relerr(_refined(tdm, dev, s.a, s.b, F32), ref) <= TOL
    # one row more takes the two-level scheme (segments and a reduced system of separator values)
    s2 = workloads.random_dominant(seed=10, n=n + 1, N=4)
    F2 = s2.F.astype(np.float32)
    ref2 = oracle.solve_hi(s2.a, s2.b, F2.astype(np.float64))
    assert relerr(_refined(tdm, dev, s2.a, s2.b, F2), ref2) <= TOL


@pytest.mark.parametrize("n,N", [(12289, 37), (16384, 300)])
def test_cooperative_launch_matches_clusters(tdm, dev, oracle, n, N):
    """Plans that need clusters of 13 to 16 CTAs solve in a cooperative launch
    (CTA groups exchanging through global memory).  The same plan solved with
    clusters -- the per-series batched layout never uses the cooperative
    launch -- gives the same result bit for bit, and it meets the gate; a CUDA
    graph that captured the cooperative solve replays it exactly."""
    from paper_0901_2859_gb300 import workloads
    s = workloads.precision(seed=5, n=n, N=N, s=1e-6)
    plan = tdm.prepare(s.a, s.b, device=dev)
    F = torch.from_numpy(s.F).to(dev)
    Xc = plan.solve(F, "fp32_refined")
    tdm.set_batched_strategy("per_series")
    try:
        Xk = tdm.solve_batched([plan], [F], "fp32_refined")[0]
    finally:
        tdm.set_batched_strategy("auto")
    torch.cuda.synchronize()
    assert torch.equal(Xc, Xk)
    cols = np.r_[0:4, N - 4:N]
    ref = oracle.solve_hi(s.a, s.b, np.ascontiguousarray(s.F[:, cols], dtype=np.float64))
    assert relerr(Xc[:, cols].cpu().numpy(), ref) <= TOL
    out = torch.empty_like(Xc)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        plan.solve(F, "fp32_refined", out=out)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.solve(F, "fp32_refined", out=out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, Xc)
    assert plan.info()["device_error"] == 0
    plan.close()
