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
