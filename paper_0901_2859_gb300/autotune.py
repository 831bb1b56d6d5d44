"""Measured choice of a matrix's solve configuration.

Two parameters shape the solve kernels:

* ``block_rows``: rows per block, 16 or 32. This is the size of the paper's
  subvectors, and it fixes M and the length of the separator recurrences.
* ``tile_rhs``: right-hand sides per tile of the refined kernel, 4, 8 or 16.
  It fixes how many blocks a CTA owns and the cluster size.

``tune`` times every valid combination on a sample block of right-hand sides
with CUDA events and keeps the fastest. It caches the choice per (device,
n, precision) in a JSON file: ``$TDM_TUNE_CACHE``, else
``~/.cache/tdm/autotune.json``. ``prepare_tuned`` prepares a plan with the
cached or measured choice. The library's own rule (32 rows; 8 right-hand
sides, or 16 where 8 would need exactly 8 or 16 CTAs per tile) is the default
without tuning.

For batches of many matrices (the per-mode series of Section 4):

* ``tune_size_classes`` tunes the tile width once per size class (the
  matrices whose n lies in one power-of-two octave), on the largest matrix of
  the class, with 32-row blocks (a batched call needs one block size);
  ``prepare_batch`` prepares every matrix with its class's choice, so the
  batched work list is built from tuned tile shapes;
* ``tune_layout`` times the batched layouts (``set_batched_strategy``) on the
  caller's own batch, caches the fastest per (device, batch signature) and
  selects it.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from .api import TDMError, prepare, set_batched_strategy, solve_batched

__all__ = ["CANDIDATES", "PLAIN_CANDIDATES", "BATCH_TILES", "LAYOUTS", "cache_path", "tune", "prepare_tuned",
           "select", "size_class", "tune_size_classes", "prepare_batch", "batch_signature", "tune_layout"]

# (block_rows, tile_rhs); tile_rhs only changes the refined kernel
CANDIDATES = ((32, 8), (32, 16), (32, 4), (16, 8), (16, 4))
PLAIN_CANDIDATES = ((32, 0), (16, 0))
# tile widths a batch's size classes choose from (a batched call needs one block size)
BATCH_TILES = ((32, 8), (32, 16), (32, 4))
# the batched layouts (set_batched_strategy), the rule's choices first
LAYOUTS = ("per_series", "by_width", "cooperative", "grouped")
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("TDM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "tdm", "autotune.json")


def _key(device_name: str, n: int, precision: str) -> str:
    return f"{device_name}|n={n}|{precision}"


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _write(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def select(candidates, measure):
    """The candidate with the smallest measured time. measure(c) returns a time,
    or None when the configuration does not apply (e.g. does not fit the size)."""
    times = {}
    for c in candidates:
        t = measure(c)
        if t is not None:
            times[c] = float(t)
    if not times:
        raise ValueError("no candidate configuration applies")
    best = min(times, key=lambda c: (times[c], candidates.index(c)))
    return best, times


def _measure(a, b, dev, precision, block_rows, tile_rhs, sample_rhs, reps):
    try:
        plan = prepare(a, b, block_rows=block_rows, tile_rhs=tile_rhs, device=dev)
    except TDMError:
        return None
    try:
        n = plan.n
        gen = torch.Generator(device=dev)
        gen.manual_seed(n)
        dt_in = torch.float64 if precision == "fp64" else torch.float32
        F = torch.randn((n, sample_rhs), device=dev, generator=gen, dtype=torch.float32).to(dt_in)
        X = torch.empty((n, sample_rhs), device=dev, dtype=torch.float32 if precision == "fp32" else torch.float64)
        plan.solve(F, precision, out=X)   # warm-up (and first-use set-up)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.solve(F, precision, out=X)
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps
    except TDMError:
        return None
    finally:
        plan.close()


def tune(a, b, precision: str = "fp32_refined", device=None, sample_rhs: int = 2048, reps: int = 3,
         use_cache: bool = True, candidates=None) -> dict:
    """{'block_rows', 'tile_rhs', 'ms', 'candidates'} for the matrix (a, b)."""
    if candidates is None:
        candidates = CANDIDATES if precision == "fp32_refined" else PLAIN_CANDIDATES
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    n = int(len(b))
    key = _key(torch.cuda.get_device_name(dev), n, precision)
    path = cache_path()
    with _lock:
        if use_cache:
            hit = _read(path).get(key)
            if hit:
                return hit
        best, times = select(list(candidates),
                             lambda c: _measure(a, b, dev, precision, c[0], c[1], sample_rhs, reps))
        entry = {"block_rows": best[0], "tile_rhs": best[1], "ms": times[best], "sample_rhs": sample_rhs,
                 "candidates": {f"{c[0]}x{c[1]}": t for c, t in times.items()}}
        if use_cache:
            data = _read(path)
            data[key] = entry
            _write(path, data)
        return entry


def prepare_tuned(a, b, precision: str = "fp32_refined", device=None, **tune_kw):
    """prepare() with the tuned block_rows and tile_rhs of this size."""
    cfg = tune(a, b, precision=precision, device=device, **tune_kw)
    return prepare(a, b, block_rows=cfg["block_rows"], tile_rhs=cfg["tile_rhs"], device=device)


def size_class(n: int) -> int:
    """The octave of n: matrices with 2^k <= n < 2^(k+1) share class k."""
    return int(n).bit_length() - 1


def tune_size_classes(series, precision: str = "fp32_refined", device=None, sample_rhs: int = 1024,
                      reps: int = 3, use_cache: bool = True) -> dict:
    """{class: tile_rhs} for the (a, b) pairs of ``series``: each class's width
    measured (or read from the cache) on its largest matrix."""
    rep = {}
    for a, b in series:
        k = size_class(len(b))
        if k not in rep or len(b) > len(rep[k][1]):
            rep[k] = (a, b)
    out = {}
    for k, (a, b) in sorted(rep.items()):
        cfg = tune(a, b, precision=precision, device=device, sample_rhs=sample_rhs, reps=reps,
                   use_cache=use_cache, candidates=BATCH_TILES)
        out[k] = cfg["tile_rhs"]
    return out


def prepare_batch(series, precision: str = "fp32_refined", device=None, **tune_kw):
    """Plans for the (a, b) pairs of ``series``, each with its size class's
    tuned tile width (32-row blocks)."""
    tiles = tune_size_classes(series, precision=precision, device=device, **tune_kw)
    return [prepare(a, b, block_rows=32, tile_rhs=tiles[size_class(len(b))], device=device) for a, b in series]


def batch_signature(plans, Fs) -> str:
    """The sizes a batched call sees: (n, right-hand sides, tile width) of every
    series, in order, hashed."""
    import hashlib
    h = hashlib.sha256()
    for p, F in zip(plans, Fs):
        h.update(f"{p.n},{int(F.shape[1])},{p.info()['tile_rhs']};".encode())
    return h.hexdigest()[:16]


def tune_layout(plans, Fs, outs, precision: str = "fp32_refined", reps: int = 3, use_cache: bool = True,
                layouts=LAYOUTS) -> dict:
    """Time ``solve_batched(plans, Fs, outs=outs)`` under each batched layout,
    select the fastest (process-wide, ``set_batched_strategy``) and cache it
    per (device, batch signature).  Returns {'layout', 'ms', 'layouts'}."""
    dev = Fs[0].device
    key = f"{torch.cuda.get_device_name(dev)}|batch={batch_signature(plans, Fs)}|{precision}"
    path = cache_path()
    with _lock:
        if use_cache:
            hit = _read(path).get(key)
            if hit:
                set_batched_strategy(hit["layout"])
                return hit

        def measure(layout):
            set_batched_strategy(layout)
            try:
                solve_batched(plans, Fs, precision, outs=outs)   # builds the layout's work list
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    solve_batched(plans, Fs, precision, outs=outs)
                e1.record()
                torch.cuda.synchronize(dev)
                return e0.elapsed_time(e1) / reps
            except TDMError:
                return None

        try:
            best, times = select(list(layouts), measure)
        finally:
            set_batched_strategy("auto")
        set_batched_strategy(best)
        entry = {"layout": best, "ms": times[best], "layouts": times}
        if use_cache:
            data = _read(path)
            data[key] = entry
            _write(path, data)
        return entry
