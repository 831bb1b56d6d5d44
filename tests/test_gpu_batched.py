"""Batched solves: many distinct matrices of uneven size in one call (the
Fourier-mode series of Section 4), checked against the oracle and against one
solve per matrix; the call is captured in a CUDA graph and replayed."""
import numpy as np
import pytest
import torch

from helpers import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdm():
    import paper_0901_2859_gb300 as m
    return m


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    return torch.device("cuda", 0)


def _batch(seed, count, n_min, n_max, N_max):
    from paper_0901_2859_gb300 import workloads
    return workloads.batching(seed=seed, count=count, K=count, n_median=int(np.sqrt(n_min * n_max)),
                              n_min=n_min, n_max=n_max, N_max=N_max)


def _upload(tdm, dev, series):
    plans = [tdm.prepare(s.a, s.b, device=dev) for s in series]
    Fs = [torch.from_numpy(s.F).to(dev) for s in series]
    return plans, Fs


def test_batched_refined_matches_oracle_and_single_solves(tdm, dev, oracle):
    series = _batch(seed=0, count=24, n_min=64, n_max=6000, N_max=70)
    plans, Fs = _upload(tdm, dev, series)
    Xb = tdm.solve_batched(plans, Fs, "fp32_refined")
    Xs = [p.solve(F, "fp32_refined") for p, F in zip(plans, Fs)]
    torch.cuda.synchronize()
    for s, xb, xs in zip(series, Xb, Xs):
        assert torch.equal(xb, xs)
        ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
        assert relerr(xb.cpu().numpy(), ref) <= 1e-11
    assert plans[0].info()["device_error"] == 0
    for p in plans:
        p.close()


def test_batched_large_and_small_sizes(tdm, dev, oracle):
    """Sizes from 256 to 40000 rows (cluster widths 1..16) in one call."""
    from paper_0901_2859_gb300 import workloads
    sizes = [(256, 5), (1000, 3), (3000, 17), (9000, 9), (20000, 4), (40000, 8)]
    series = []
    for m, (n, N) in enumerate(sizes):
        rng = np.random.default_rng(m)
        s = 4.0 * np.sin(np.pi * (m + 1) / (2.0 * 513)) ** 2
        series.append(workloads.Series(-np.ones(n - 1), np.full(n, 2.0 + s),
                                       rng.standard_normal((n, N), dtype=np.float32)))
    plans, Fs = _upload(tdm, dev, series)
    Xb = tdm.solve_batched(plans, Fs, "fp32_refined")
    torch.cuda.synchronize()
    for s, xb in zip(series, Xb):
        ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
        assert relerr(xb.cpu().numpy(), ref) <= 1e-11, s.n
    for p in plans:
        p.close()


def test_batched_call_replays_in_a_cuda_graph(tdm, dev):
    series = _batch(seed=1, count=16, n_min=128, n_max=4000, N_max=40)
    plans, Fs = _upload(tdm, dev, series)
    outs = [torch.empty((p.n, F.shape[1]), dtype=torch.float64, device=dev) for p, F in zip(plans, Fs)]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        tdm.solve_batched(plans, Fs, "fp32_refined", outs=outs)   # builds the work list
    torch.cuda.synchronize()
    ref = [x.clone() for x in outs]
    for x in outs:
        x.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        tdm.solve_batched(plans, Fs, "fp32_refined", outs=outs)
    graph.replay()
    torch.cuda.synchronize()
    for x, r in zip(outs, ref):
        assert torch.equal(x, r)
    for F in Fs:   # new right-hand sides in place, replay again
        F.mul_(2.0)
    graph.replay()
    torch.cuda.synchronize()
    for x, r in zip(outs, ref):
        assert torch.allclose(x, 2.0 * r, rtol=1e-12, atol=0)
    for p in plans:
        p.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_other_precisions(tdm, dev, oracle, precision):
    series = _batch(seed=2, count=6, n_min=100, n_max=3000, N_max=20)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plans = [tdm.prepare(s.a, s.b, device=dev) for s in series]
    Fs = [torch.from_numpy(s.F).to(dev, dt) for s in series]
    Xb = tdm.solve_batched(plans, Fs, precision)
    torch.cuda.synchronize()
    for s, xb in zip(series, Xb):
        ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
        assert relerr(xb.cpu().numpy(), ref) <= (1e-11 if precision == "fp64" else 2e-5)
    for p in plans:
        p.close()


@pytest.fixture(params=["grouped", "cooperative"])
def grouped(tdm, request):
    """The layouts in which tiles of several series share one launch."""
    tdm.set_batched_strategy(request.param)
    yield request.param
    tdm.set_batched_strategy("auto")


@pytest.mark.parametrize("strategy", ["per_series", "by_width", "grouped", "cooperative"])
def test_batched_strategies_match_single_solves(tdm, dev, oracle, strategy):
    """Both layouts of the batched work give every series the result of its own
    solve, bit for bit, over sizes that need clusters of 1 to 16 CTAs and
    three kernel shapes (up to n = 40000)."""
    sizes = [(300, 9), (700, 30), (2100, 17), (5000, 8), (9000, 21), (15000, 5), (20000, 6), (40000, 3)]
    from paper_0901_2859_gb300 import workloads
    series = []
    for m, (n, N) in enumerate(sizes):
        rng = np.random.default_rng(40 + m)
        s = 4.0 * np.sin(np.pi * (m + 1) / (2.0 * 65)) ** 2
        series.append(workloads.Series(-np.ones(n - 1), np.full(n, 2.0 + s),
                                       rng.standard_normal((n, N), dtype=np.float32)))
    plans, Fs = _upload(tdm, dev, series)
    tdm.set_batched_strategy(strategy)
    try:
        Xb = tdm.solve_batched(plans, Fs, "fp32_refined")
    finally:
        tdm.set_batched_strategy("auto")
    Xs = [p.solve(F, "fp32_refined") for p, F in zip(plans, Fs)]
    torch.cuda.synchronize()
    for s, xb, xs in zip(series, Xb, Xs):
        assert torch.equal(xb, xs), s.n
    ref = oracle.solve_hi(series[4].a, series[4].b, series[4].F.astype(np.float64))
    assert relerr(Xb[4].cpu().numpy(), ref) <= 1e-11
    for p in plans:
        assert p.info()["device_error"] == 0
        p.close()


def test_grouped_launch_mixed_schedules(tdm, dev, oracle, grouped):
    """Plans of three correction schedules in one call -- the calibrated
    per-tile test, two fixed corrections, the uncalibrated test.  Grouped
    units put each schedule in a launch of its own; the first two equal the
    plan's own solve bit for bit (a series keeps its single-series partition
    inside its group), the third runs the fixed retry count.  Cooperative runs
    mix them in one launch and all three equal the plan's own solve.  All meet
    the gate."""
    series = _batch(seed=5, count=18, n_min=100, n_max=9000, N_max=50)
    steps = [0, 2, -1] * 6
    plans = [tdm.prepare(s.a, s.b, refine_steps=k, device=dev) for s, k in zip(series, steps)]
    Fs = [torch.from_numpy(s.F).to(dev) for s in series]
    Xb = tdm.solve_batched(plans, Fs, "fp32_refined")
    Xs = [p.solve(F, "fp32_refined") for p, F in zip(plans, Fs)]
    torch.cuda.synchronize()
    for s, k, xb, xs in zip(series, steps, Xb, Xs):
        if k != -1 or grouped == "cooperative":
            assert torch.equal(xb, xs), (s.n, k)
        ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
        assert relerr(xb.cpu().numpy(), ref) <= 1e-11, (s.n, k)
    for p in plans:
        assert p.info()["device_error"] == 0
        p.close()


def test_grouped_launch_retries_a_failing_unit(tdm, dev, oracle, grouped):
    """Pure high sine modes at kappa ~ 3.4e6 (n = 4096, a group of 4 CTAs) need
    more than one correction: the speculative test fails on their units, and
    the cluster solves each such unit again with the fixed retry count --
    together with the tiles of the other series that shared the unit (a
    16-CTA series sets the cluster width, 1-CTA series fill the gaps).
    Everything meets its gate and no tile reports non-convergence."""
    from paper_0901_2859_gb300 import workloads
    s4 = workloads.poisson2d(seed=1)
    n = s4.n
    ks = [n // 2, n - 1, n] * 6
    Fe, _, lam = oracle.eigen_closed_form(n, s4.b[0], ks)
    lam_min = oracle.eigen_closed_form(n, s4.b[0], [1])[2][0]
    series = [workloads.Series(s4.a, s4.b, Fe.astype(np.float32))]
    tols = [[max(1e-11, 0.1 * 2.0 ** -48 * np.sqrt(lam[c]) / lam_min) for c in range(len(ks))]]
    big = workloads.precision(seed=2, n=16384, N=24, s=1e-6)
    series.append(big)
    tols.append([1e-11] * big.F.shape[1])
    for m in range(10):
        rng = np.random.default_rng(100 + m)
        nn = int(rng.integers(200, 1000))
        sh = 4.0 * np.sin(np.pi * (m + 1) / (2.0 * 513)) ** 2
        series.append(workloads.Series(-np.ones(nn - 1), np.full(nn, 2.0 + sh),
                                       rng.standard_normal((nn, 40), dtype=np.float32)))
        tols.append([1e-11] * 40)
    plans, Fs = _upload(tdm, dev, series)
    Xb = tdm.solve_batched(plans, Fs, "fp32_refined")
    torch.cuda.synchronize()
    for s, tol, xb in zip(series, tols, Xb):
        ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
        x = xb.cpu().numpy()
        errs = [relerr(x[:, c], ref[:, c]) for c in range(x.shape[1])]
        assert all(e <= t for e, t in zip(errs, tol)), (s.n, max(errs))
    for p in plans:
        assert p.info()["device_error"] == 0
        p.close()


@pytest.mark.parametrize("strategy", ["auto", "cooperative"])
def test_batching_workload_sampled_against_the_oracle(tdm, dev, oracle, strategy):
    """The full batching workload (512 Fourier-mode matrices of lognormal size
    up to n = 43943, 1.7e9 unknowns, F ~ N(0,1) drawn on the device) in one
    call, as the benchmark runs it; sampled columns of 16 matrices (the three
    largest and 13 others) against the oracle's solve."""
    from paper_0901_2859_gb300 import workloads
    specs = workloads.batching(seed=0, rhs=False)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    plans = [tdm.prepare(s.a, s.b, device=dev) for s in specs]
    Fs = [torch.randn((s.n, s.meta["N"]), device=dev, dtype=torch.float32, generator=gen) for s in specs]
    tdm.set_batched_strategy(strategy)
    try:
        Xs = tdm.solve_batched(plans, Fs, "fp32_refined")
    finally:
        tdm.set_batched_strategy("auto")
    torch.cuda.synchronize()
    order = np.argsort([s.n for s in specs])
    rng = np.random.default_rng(7)
    pick = list(order[-3:]) + list(rng.choice(order[:-3], size=13, replace=False))
    for k in pick:
        s, N = specs[k], specs[k].meta["N"]
        cols = np.unique(np.r_[0, N - 1, rng.integers(0, N, size=2)])
        F = Fs[k][:, cols].cpu().numpy().astype(np.float64)
        ref = oracle.solve_hi(s.a, s.b, F)
        assert relerr(Xs[k][:, cols].cpu().numpy(), ref) <= 1e-11, (k, s.n, N)
    assert all(p.info()["device_error"] == 0 for p in plans)
    for p in plans:
        p.close()


def test_batched_refined_with_a_plan_beyond_one_cluster(tdm, dev, oracle):
    """A batch whose largest series (n = 70001) needs the two-level solve: it is
    solved by that solve inside the same call, the others by the batched layout;
    everything meets the gate and equals the series' own solves."""
    from paper_0901_2859_gb300 import workloads
    sizes = [(70001, 6), (3000, 20), (900, 9)]
    series = []
    for m, (n, N) in enumerate(sizes):
        rng = np.random.default_rng(70 + m)
        sh = 4.0 * np.sin(np.pi * (m + 1) / (2.0 * 65)) ** 2
        series.append(workloads.Series(-np.ones(n - 1), np.full(n, 2.0 + sh),
                                       rng.standard_normal((n, N), dtype=np.float32)))
    plans, Fs = _upload(tdm, dev, series)
    Xb = tdm.solve_batched(plans, Fs, "fp32_refined")
    Xs = [p.solve(F, "fp32_refined") for p, F in zip(plans, Fs)]
    torch.cuda.synchronize()
    for s, xb, xs in zip(series, Xb, Xs):
        assert torch.equal(xb, xs), s.n
        ref = oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))
        assert relerr(xb.cpu().numpy(), ref) <= 1e-11, s.n
    for p in plans:
        assert p.info()["device_error"] == 0
        p.close()
