"""tdm_solve_batched_noalloc, called through the C ABI: the batched refined
solve whose work list lives in a fixed device array of the library (the call
allocates nothing).  Two different batches are solved in a row -- the second
call overwrites the array the first one filled -- and both are compared with
tdm_solve_batched and with the oracle.  The file is collected last, and passes
alone or after every other test."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import relerr

pytestmark = pytest.mark.gpu

TOL = 1e-11                      # the refined path's gate in every other test
TDM_ERR_TOO_LARGE = 8


@pytest.fixture(scope="module")
def env():
    assert torch.cuda.is_available()
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import _lib
    return tdm, _lib.load(), torch.device("cuda", 0)


def _call(lib, plans, Fs, outs, dev):
    """Marshal the arguments and call the C entry point directly."""
    count = len(plans)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    hs = (vp * count)(*[p.handle.value for p in plans])
    fp = (vp * count)(*[F.data_ptr() for F in Fs])
    xp = (vp * count)(*[X.data_ptr() for X in outs])
    ldf = (i64 * count)(*[F.stride(0) for F in Fs])
    ldx = (i64 * count)(*[X.stride(0) for X in outs])
    ns = (i64 * count)(*[F.shape[1] for F in Fs])
    stream = vp(torch.cuda.current_stream(dev).cuda_stream)
    return lib.tdm_solve_batched_noalloc(hs, count, fp, ldf, xp, ldx, ns, stream)


def _batch(tdm, dev, seed, count, n_min, n_max, N_max):
    from paper_0901_2859_gb300 import workloads
    series = workloads.batching(seed=seed, count=count, K=count, n_median=int(np.sqrt(n_min * n_max)),
                                n_min=n_min, n_max=n_max, N_max=N_max)
    plans = [tdm.prepare(s.a, s.b, device=dev) for s in series]
    Fs = [torch.from_numpy(s.F).to(dev) for s in series]
    return series, plans, Fs


def _nan_outs(plans, Fs, dev):
    return [torch.full((p.n, F.shape[1]), float("nan"), dtype=torch.float64, device=dev)
            for p, F in zip(plans, Fs)]


def test_two_calls_in_a_row_match_batched_and_oracle(env, oracle):
    tdm, lib, dev = env
    sA, pA, FA = _batch(tdm, dev, seed=21, count=12, n_min=64, n_max=6000, N_max=70)
    sB, pB, FB = _batch(tdm, dev, seed=22, count=7, n_min=200, n_max=20000, N_max=40)
    refA = tdm.solve_batched(pA, FA, "fp32_refined")
    refB = tdm.solve_batched(pB, FB, "fp32_refined")
    outA, outB, outA2 = _nan_outs(pA, FA, dev), _nan_outs(pB, FB, dev), _nan_outs(pA, FA, dev)
    torch.cuda.synchronize()
    assert _call(lib, pA, FA, outA, dev) == 0      # the first call on the device sets it up
    assert _call(lib, pB, FB, outB, dev) == 0      # overwrites the work list of the first
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    assert _call(lib, pA, FA, outA2, dev) == 0     # the array still holds the second call's items
    assert _call(lib, pB, FB, outB, dev) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0   # no device memory taken by the calls
    for series, outs, refs in ((sA, outA, refA), (sB, outB, refB), (sA, outA2, refA)):
        for s, x, r in zip(series, outs, refs):
            xn = x.cpu().numpy()
            assert np.isfinite(xn).all()
            assert relerr(xn, r.cpu().numpy()) <= TOL
            assert relerr(xn, oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))) <= TOL
    assert pA[0].info()["device_error"] == 0
    assert pB[0].info()["device_error"] == 0
    for p in pA + pB:
        p.close()


def test_capacity_limit(env, oracle):
    """A 64-row system takes 8 right-hand sides per tile: 8 * 4096 columns fill
    the array exactly; one more column is rejected before anything runs."""
    tdm, lib, dev = env
    from paper_0901_2859_gb300 import _lib
    n, cap = 64, _lib.NOALLOC_MAX_TILES
    rng = np.random.default_rng(5)
    a, b = -np.ones(n - 1), np.full(n, 2.0 + 1e-3)
    plan = tdm.prepare(a, b, device=dev)
    F = torch.from_numpy(rng.standard_normal((n, 8 * cap + 1), dtype=np.float32)).to(dev)
    full = F[:, :8 * cap]
    X = torch.full((n, 8 * cap + 1), float("nan"), dtype=torch.float64, device=dev)
    assert _call(lib, [plan], [F], [X], dev) == TDM_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.isnan(X).all()                    # nothing was enqueued
    Xf = X[:, :8 * cap]
    assert _call(lib, [plan], [full], [Xf], dev) == 0
    ref = plan.solve(full.contiguous(), "fp32_refined")
    torch.cuda.synchronize()
    assert relerr(Xf.cpu().numpy(), ref.cpu().numpy()) <= TOL
    cols = [0, 1, 4095, 8 * cap - 1]
    ora = oracle.solve_hi(a, b, F[:, cols].cpu().numpy().astype(np.float64))
    assert relerr(Xf[:, cols].cpu().numpy(), ora) <= TOL
    plan.close()


TDM_ERR_NOT_IMPLEMENTED = 7


def test_refused_under_stream_capture(env):
    """Under stream capture the call returns TDM_ERR_NOT_IMPLEMENTED and enqueues
    nothing: a captured copy of the host-side work list would be re-read at every
    replay, after later calls have refilled it."""
    tdm, lib, dev = env
    _, plans, Fs = _batch(tdm, dev, seed=23, count=3, n_min=100, n_max=3000, N_max=20)
    outs = _nan_outs(plans, Fs, dev)
    marker = torch.zeros(4, device=dev)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        marker.add_(1.0)                            # the graph is not empty
        status = _call(lib, plans, Fs, outs, dev)
    assert status == TDM_ERR_NOT_IMPLEMENTED
    graph.replay()
    torch.cuda.synchronize()
    assert all(torch.isnan(x).all() for x in outs)  # no solve was captured
    assert float(marker[0]) == 1.0
    for p in plans:
        p.close()


def test_calls_on_two_streams_ordered_by_an_event(env, oracle):
    """Call A on one stream, an event makes a second stream wait for it, call B
    (which overwrites the shared work list) on the second stream: both right."""
    tdm, lib, dev = env
    sA, pA, FA = _batch(tdm, dev, seed=24, count=5, n_min=64, n_max=5000, N_max=30)
    sB, pB, FB = _batch(tdm, dev, seed=25, count=6, n_min=300, n_max=9000, N_max=50)
    outA, outB = _nan_outs(pA, FA, dev), _nan_outs(pB, FB, dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    s1.wait_stream(torch.cuda.current_stream(dev))
    s2.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s1):
        assert _call(lib, pA, FA, outA, dev) == 0
    done_a = torch.cuda.Event()
    done_a.record(s1)
    s2.wait_event(done_a)
    with torch.cuda.stream(s2):
        assert _call(lib, pB, FB, outB, dev) == 0
    torch.cuda.synchronize()
    for series, outs in ((sA, outA), (sB, outB)):
        for s, x in zip(series, outs):
            xn = x.cpu().numpy()
            assert np.isfinite(xn).all()
            assert relerr(xn, oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))) <= TOL
    for p in pA + pB:
        p.close()
