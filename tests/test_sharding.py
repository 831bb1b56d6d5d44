"""Right-hand-side sharding across ranks, on CPU with the gloo backend and two
processes: every rank solves its own columns (here with the oracle's sweep,
which stands in for the GPU solve), the shards reassemble into the solution of
the whole series, and the timing reduction takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0901_2859_gb300.sharding import gather_columns, max_over_ranks, shard_columns


@pytest.mark.parametrize("N,world", [(0, 2), (1, 2), (7, 2), (8, 3), (64, 5), (3, 8)])
def test_shards_cover_every_column_once(N, world):
    ranges = [shard_columns(N, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == N
    for (s0, e0), (s1, _) in zip(ranges, ranges[1:]):
        assert e0 == s1
    sizes = [e - s for s, e in ranges]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == N


def test_bad_rank_rejected():
    with pytest.raises(ValueError):
        shard_columns(10, 2, 2)
    with pytest.raises(ValueError):
        shard_columns(-1, 2, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, N, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_0901_2859_gb300 import workloads
        s = workloads.plain_fp64(seed=3, n=n, N=N)   # every rank draws the same series
        start, stop = shard_columns(N, world, rank)
        X_local = torch.from_numpy(oracle.thomas_f64(s.a, s.b, np.ascontiguousarray(s.F[:, start:stop]), threads=1))
        X = gather_columns(X_local, N)
        slowest = max_over_ranks(float(rank + 1))
        if rank == 0:
            np.savez(result_path, X=X.numpy(), slowest=slowest)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_series(tmp_path, oracle):
    n, N, world = 300, 37, 2
    out = str(tmp_path / "x.npz")
    mp.start_processes(_rank_main, args=(world, _free_port(), n, N, out), nprocs=world, join=True,
                       start_method="spawn")
    from paper_0901_2859_gb300 import workloads
    s = workloads.plain_fp64(seed=3, n=n, N=N)
    res = np.load(out)
    ref = oracle.thomas_f64(s.a, s.b, s.F)
    assert np.array_equal(res["X"], ref)    # the same sweep on the same columns: bit-identical
    assert float(res["slowest"]) == float(world)
