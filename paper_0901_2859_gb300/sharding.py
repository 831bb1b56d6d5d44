"""Right-hand-side sharding across ranks (one process per GPU).

Every column of a series A X = F is independent once the matrix is prepared
(the per-right-hand-side step of Algorithms 3 and 4 reads nothing but its own
column and the plan), so a series is split by columns: each rank prepares its
own copy of the plan and solves a contiguous range of columns.  No collective
is needed in the data path; ``gather_columns`` exists for a caller that wants
the whole X on every rank, and ``max_over_ranks`` is the timing reduction the
benchmark uses.
"""
from __future__ import annotations

import torch

__all__ = ["shard_columns", "max_over_ranks", "gather_columns"]


def shard_columns(N: int, world: int, rank: int) -> tuple[int, int]:
    """Columns [start, stop) of rank `rank` when N columns are split over
    `world` ranks as evenly as possible (the first N % world ranks get one
    more)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError(f"bad rank {rank} of {world}")
    if N < 0:
        raise ValueError("N must be >= 0")
    base, extra = divmod(N, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(x: float, group=None, device=None) -> float:
    """The largest x over the ranks of `group` (x itself without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_columns(X_local: torch.Tensor, N: int, group=None) -> torch.Tensor:
    """Reassemble the (n, N) solution from every rank's (n, stop - start) shard."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = X_local.shape[0]
    widest = max(stop - start for start, stop in (shard_columns(N, world, r) for r in range(world)))
    pad = torch.zeros((n, widest), dtype=X_local.dtype, device=X_local.device)
    pad[:, :X_local.shape[1]] = X_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad.contiguous(), group=group)
    out = torch.empty((n, N), dtype=X_local.dtype, device=X_local.device)
    for r, part in enumerate(parts):
        start, stop = shard_columns(N, world, r)
        out[:, start:stop] = part[:, :stop - start]
    return out
