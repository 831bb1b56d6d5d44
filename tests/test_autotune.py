"""The configuration autotuner: the selection and its JSON cache on CPU (with a
fake timer), and a tuned plan on the GPU checked against the oracle."""
import json

import numpy as np
import pytest

from helpers import relerr


def test_select_takes_the_fastest_applicable_candidate():
    from paper_0901_2859_gb300.autotune import select
    times = {(32, 8): 2.0, (32, 16): 1.5, (32, 4): None, (16, 8): 1.5}
    best, measured = select(list(times), times.get)
    assert best == (32, 16)            # ties go to the earlier candidate
    assert (32, 4) not in measured and measured[(16, 8)] == 1.5
    with pytest.raises(ValueError):
        select([(32, 8)], lambda c: None)


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_0901_2859_gb300 import autotune
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("TDM_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    autotune._write(str(path), {"k": {"block_rows": 16}})
    assert autotune._read(str(path)) == {"k": {"block_rows": 16}}
    path.write_text("not json")
    assert autotune._read(str(path)) == {}


@pytest.mark.gpu
def test_tuned_plan_matches_oracle_and_is_cached(tmp_path, monkeypatch, oracle):
    import torch
    from paper_0901_2859_gb300 import autotune, workloads
    monkeypatch.setenv("TDM_TUNE_CACHE", str(tmp_path / "tune.json"))
    dev = torch.device("cuda", 0)
    s = workloads.precision(seed=2, n=3000, N=40, s=1e-4)
    cfg = autotune.tune(s.a, s.b, device=dev, sample_rhs=64, reps=2)
    assert (cfg["block_rows"], cfg["tile_rhs"]) in autotune.CANDIDATES
    assert len(cfg["candidates"]) >= 2
    cached = json.loads((tmp_path / "tune.json").read_text())
    assert list(cached.values())[0]["block_rows"] == cfg["block_rows"]
    monkeypatch.setattr(autotune, "_measure", lambda *a, **k: pytest.fail("cache not used"))
    plan = autotune.prepare_tuned(s.a, s.b, device=dev, sample_rhs=64, reps=2)
    assert plan.info()["block_rows"] == cfg["block_rows"] and plan.info()["tile_rhs"] == cfg["tile_rhs"]
    X = plan.solve(torch.from_numpy(s.F).to(dev), "fp32_refined")
    torch.cuda.synchronize()
    assert relerr(X.cpu().numpy(), oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))) <= 1e-11
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [4, 8, 16])
def test_requested_tile_widths_agree(tile, oracle):
    import torch
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    dev = torch.device("cuda", 0)
    s = workloads.precision(seed=3, n=5000, N=37, s=1e-5)
    plan = tdm.prepare(s.a, s.b, tile_rhs=tile, device=dev)
    assert plan.info()["tile_rhs"] == tile
    X = plan.solve(torch.from_numpy(s.F).to(dev), "fp32_refined")
    torch.cuda.synchronize()
    assert relerr(X.cpu().numpy(), oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))) <= 1e-11
    plan.close()


def test_size_classes_are_octaves():
    from paper_0901_2859_gb300.autotune import size_class
    assert [size_class(n) for n in (1, 2, 3, 1023, 1024, 2047, 16384)] == [0, 1, 1, 9, 10, 10, 14]


@pytest.mark.gpu
def test_batch_tuning_per_size_class_and_layout(tmp_path, monkeypatch, oracle):
    """A batch of 12 matrices over three octaves: one tile width tuned per
    class on its largest matrix, the plans built with them, the batched layouts
    timed on the batch and the fastest selected and cached; the tuned batch
    meets the gate against the oracle."""
    import torch
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import autotune, workloads
    monkeypatch.setenv("TDM_TUNE_CACHE", str(tmp_path / "tune.json"))
    dev = torch.device("cuda", 0)
    specs = workloads.batching(seed=3, count=12, K=12, n_median=2000, n_min=700, n_max=6000, N_max=60)
    pairs = [(s.a, s.b) for s in specs]
    tiles = autotune.tune_size_classes(pairs, device=dev, sample_rhs=64, reps=2)
    assert set(tiles) == {autotune.size_class(len(b)) for _, b in pairs}
    assert all(t in (4, 8, 16) for t in tiles.values())
    plans = autotune.prepare_batch(pairs, device=dev, sample_rhs=64, reps=2)
    assert [p.info()["tile_rhs"] for p in plans] == [tiles[autotune.size_class(p.n)] for p in plans]
    Fs = [torch.from_numpy(s.F).to(dev) for s in specs]
    outs = [torch.empty((p.n, F.shape[1]), dtype=torch.float64, device=dev) for p, F in zip(plans, Fs)]
    try:
        choice = autotune.tune_layout(plans, Fs, outs, reps=2)
        assert choice["layout"] in autotune.LAYOUTS and len(choice["layouts"]) == len(autotune.LAYOUTS)
        cached = json.loads((tmp_path / "tune.json").read_text())
        assert any(v.get("layout") == choice["layout"] for v in cached.values())
        tdm.solve_batched(plans, Fs, "fp32_refined", outs=outs)
        torch.cuda.synchronize()
    finally:
        tdm.set_batched_strategy("auto")
    for s, x in zip(specs, outs):
        assert relerr(x.cpu().numpy(), oracle.solve_hi(s.a, s.b, s.F.astype(np.float64))) <= 1e-11
    for p in plans:
        p.close()
