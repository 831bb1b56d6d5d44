"""Benchmark of the GB300 dichotomy solver on the precision workload.

Workload (one "step"): one solve of the series A X_n = F_n with n = 16384
unknowns and N = 8192 right-hand sides, a_i = -1, b_i = 2 + s (s = 1e-6, the
worst conditioning of the workload's range 10^[-6, 0], kappa ~ 3.9e6), F ~ N(0,1)
in binary32, solved by the refined path (binary32 dichotomy solves + error-free
residual refinement, binary64 output) to 1e-11 relative error.  The plain
binary64 and binary32 dichotomy solves of the same series are measured beside
it.  Inputs are resident in HBM and larger than L2 (F: 512 MiB, X: 1 GiB).

Prints one JSON line (rank 0).  Multi-GPU (torchrun): every rank solves its own
N-column series (weak scaling, no collective in the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ROWS, N_RHS, SHIFT = 16384, 8192, 1e-6
METRIC = "unknowns solved/s (n*N/s) and % of HBM roofline, FP32+refine vs FP64 at 1e-11 err"
UNIT = "unknowns/s"
WORKLOAD = "precision n=16384 N=8192 s=1e-6 (a=-1, b=2+s), F~N(0,1) fp32, refined to 1e-11"
DIST = dict(rank=int(os.environ.get("RANK", 0)), world=int(os.environ.get("WORLD_SIZE", 1)),
            local=int(os.environ.get("LOCAL_RANK", 0)))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each captured kernel is built from (a capture is void once one changes)
KERNEL_SOURCES = {
    "k_refined": ("tdm_refine.cu", "tdm_refine.cuh", "tdm_f2.cuh", "tdm_df.cuh", "tdm_iface_df.cuh",
                  "tdm_kernel_common.cuh", "tdm_internal.cuh", "tdm_tma.cuh"),
}


def _kernel_hash(kernel: str = "k_refined") -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0901_2859_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t.get(kernel)
        if e and e.get("source_hash") == _kernel_hash(kernel):
            return float(e["bytes_per_launch_full"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _events_time(fn, steps: int, warmup: int, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    _barrier()
    return e0.elapsed_time(e1) / steps   # ms per call, this rank


def _barrier():
    if DIST["world"] > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, torch) -> float:
    if DIST["world"] <= 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=torch.device("cuda", DIST["local"]))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _cpu_baseline(series, cols_target: int, X_gpu_cols=None, seconds: float = 10.0):
    """The oracle's binary64 sweep on the host cores: whole passes over the first
    `cols_target` right-hand sides, repeated until `seconds` of work have passed."""
    import numpy as np
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    k = max(1, min(series.N, cols_target))
    Fs = np.ascontiguousarray(series.F[:, :k], dtype=np.float64)
    oracle.thomas_f64(series.a, series.b, Fs[:, :min(k, 8)], threads=threads)   # warm-up
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.thomas_f64(series.a, series.b, Fs, threads=threads)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    out = {"value": series.n * k * reps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"oracle binary64 sweep (thomas_f64) over {k} of {series.N} right-hand sides, n={series.n}, "
                     f"{reps} passes in {dt:.1f} s"}
    if X_gpu_cols is not None:
        idx, cols = X_gpu_cols
        ref = oracle.solve_hi(series.a, series.b, np.ascontiguousarray(series.F[:, idx], dtype=np.float64))
        den = np.maximum(np.abs(ref).max(axis=0), 1e-300)
        for name, Xg in cols.items():   # relative max-norm error per column, max over the columns
            out[f"{name}_rel_err_vs_oracle"] = float(np.max(np.abs(Xg - ref).max(axis=0) / den))
        out["error_columns"] = len(idx)
    return out


def run_gpu(args):
    N_RHS = args.rhs
    import numpy as np
    import torch
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads

    if DIST["world"] > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", DIST["local"]))
    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    series = workloads.precision(seed=DIST["rank"], n=N_ROWS, N=N_RHS, s=SHIFT)
    plan = tdm.prepare(series.a, series.b, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan2 = tdm.prepare(series.a, series.b, device=dev)
    prepare_ms = (time.perf_counter() - t0) * 1e3
    plan2.close()
    info = plan.info()
    F = torch.from_numpy(series.F).to(dev)
    X = torch.empty((N_ROWS, N_RHS), dtype=torch.float64, device=dev)
    unknowns = N_ROWS * N_RHS

    # ---- headline: refined path --------------------------------------------------------
    with ClockSampler(DIST["local"]) as clk:
        ms = _events_time(lambda: plan.solve(F, "fp32_refined", out=X), args.steps, args.warmup, torch)
    ms = _max_over_ranks(ms, torch)
    value = DIST["world"] * unknowns / (ms * 1e-3)
    hbm, peak_kind = _peaks()
    bytes_refined = unknowns * (4 + 8)
    achieved = bytes_refined / (ms * 1e-3) / 1e9
    traffic = _traffic("k_refined")

    # ---- comparison paths: plain binary64 and plain binary32 dichotomy ------------------------
    F64 = F.double()
    X32 = torch.empty((N_ROWS, N_RHS), dtype=torch.float32, device=dev)
    k64 = max(3, min(args.steps, 50))
    ms64 = _max_over_ranks(_events_time(lambda: plan.solve(F64, "fp64", out=X), k64, 2, torch), torch)
    ms32 = _max_over_ranks(_events_time(lambda: plan.solve(F, "fp32", out=X32), args.steps, args.warmup, torch), torch)
    del F64

    # ---- end to end: pinned host buffers, copies inside the timed region ----------------------
    Fh = torch.from_numpy(series.F).pin_memory()
    Xh = torch.empty((N_ROWS, N_RHS), dtype=torch.float64).pin_memory()

    def e2e_step():   # tdm_solve_host: chunked copies in and out, overlapped with the solves
        plan.solve_host(Fh, "fp32_refined", out=Xh)

    ke = max(3, min(args.steps, 20))
    ms_e2e = _max_over_ranks(_events_time(e2e_step, ke, 2, torch), torch)
    # the host link's own rates, outside the timed region: contiguous pinned copies of 256 MiB each way, and
    # 128 MiB in with 256 MiB out at the same time (the step's 1:2 ratio); the end-to-end ceiling is the step's
    # bytes at the simultaneous rate (the link does not carry both directions at their full one-way rates)
    hb = torch.empty(256 << 20, dtype=torch.uint8).pin_memory()
    db = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    hb2 = torch.empty(128 << 20, dtype=torch.uint8).pin_memory()
    db2 = torch.empty(128 << 20, dtype=torch.uint8, device=dev)
    link_h2d = (256 << 20) / (_events_time(lambda: db.copy_(hb, non_blocking=True), 3, 2, torch) * 1e-3) / 1e9
    link_d2h = (256 << 20) / (_events_time(lambda: hb.copy_(db, non_blocking=True), 3, 2, torch) * 1e-3) / 1e9
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def both_ways():
        cur = torch.cuda.current_stream(dev)
        s_in.wait_stream(cur)
        s_out.wait_stream(cur)
        with torch.cuda.stream(s_in):
            db2.copy_(hb2, non_blocking=True)
        with torch.cuda.stream(s_out):
            hb.copy_(db, non_blocking=True)
        cur.wait_stream(s_in)
        cur.wait_stream(s_out)
    link_both = (384 << 20) / (_events_time(both_ways, 3, 2, torch) * 1e-3) / 1e9
    del hb, db, hb2, db2
    ceiling_ms = unknowns * 12 / link_both / 1e6

    # the refined solution of a few columns, for the accuracy check of the baseline leg
    plan.solve(F, "fp32_refined", out=X)
    idx = np.array([0, 1, 2, 3, N_RHS // 2, N_RHS - 1])
    Xcols = {"refined": X[:, idx].cpu().numpy()}
    plan.solve(F.double(), "fp64", out=X)   # the plain binary64 path on the same columns
    Xcols["fp64"] = X[:, idx].cpu().numpy()
    dev_err = plan.info()["device_error"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": DIST["world"], "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if N_RHS == 8192 else WORKLOAD.replace("N=8192", f"N={N_RHS}"),
                   "n": N_ROWS, "N": N_RHS, "s": SHIFT, "precision": "fp32_refined",
                   "output": "f64", "refine_steps": info["refine_steps"], "contraction": info["contraction"],
                   "refinement": "one correction per tile, checked against the plan's calibrated contraction "
                                 "during the next tile; a failing tile is solved again with more",
                   "block_rows": info["block_rows"],
                   "parallelism": f"rhs-sharded x{DIST['world']}" if DIST["world"] > 1 else "single GPU",
                   "l2": f"no flush: F ({N_ROWS * N_RHS * 4 >> 20} MiB) and X ({N_ROWS * N_RHS * 8 >> 20} MiB) "
                         "exceed L2" if N_ROWS * N_RHS * 4 > (129 << 20) else "no flush: a sample smaller than L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": "k_refined", "algorithmic_bytes_per_launch": bytes_refined},
        "e2e": {"value": DIST["world"] * unknowns / (ms_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": unknowns * 4, "d2h_bytes_per_step": unknowns * 8, "ms_per_step": ms_e2e,
                "link_gbs": {"h2d": link_h2d, "d2h": link_d2h, "both_ways_1to2": link_both},
                "link_ceiling": {"value": DIST["world"] * unknowns / (ceiling_ms * 1e-3), "ms_per_step": ceiling_ms}},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "paths": {
            "fp32_refined": {"ms": ms, "unknowns_per_s": value, "hbm_frac": achieved / hbm},
            "fp64": {"ms": ms64, "unknowns_per_s": DIST["world"] * unknowns / (ms64 * 1e-3),
                     "hbm_frac": unknowns * 16 / (ms64 * 1e-3) / 1e9 / hbm},
            "fp32": {"ms": ms32, "unknowns_per_s": DIST["world"] * unknowns / (ms32 * 1e-3),
                     "hbm_frac": unknowns * 8 / (ms32 * 1e-3) / 1e9 / hbm},
            "refined_over_fp64": ms64 / ms,
        },
        "prepare_ms": prepare_ms, "device_error": dev_err,
    }
    if DIST["rank"] == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(series, args.cpu_cols, (idx, Xcols), args.cpu_seconds)
    plan.close()
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)
    if DIST["world"] > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batching(args):
    """The batching workload: 512 Fourier-mode matrices of lognormal sizes, each
    with its own right-hand sides, solved refined in one batched call (and its
    CUDA-graph replay), against one launch per matrix; the grouped-unit layout
    of the same call is timed for context."""
    import numpy as np
    import torch
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads

    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    specs = workloads.batching(seed=DIST["rank"], rhs=False)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + DIST["rank"])
    t0 = time.perf_counter()
    plans = [tdm.prepare(s.a, s.b, device=dev) for s in specs]
    torch.cuda.synchronize()
    prepare_s = time.perf_counter() - t0
    Fs = [torch.randn((s.n, s.meta["N"]), device=dev, dtype=torch.float32, generator=gen) for s in specs]
    Xs = [torch.empty((s.n, s.meta["N"]), device=dev, dtype=torch.float64) for s in specs]
    unknowns = sum(s.n * s.meta["N"] for s in specs)
    ms_batched = _events_time(lambda: tdm.solve_batched(plans, Fs, "fp32_refined", outs=Xs), args.steps, args.warmup, torch)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        tdm.solve_batched(plans, Fs, "fp32_refined", outs=Xs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        tdm.solve_batched(plans, Fs, "fp32_refined", outs=Xs)
    ms_graph = _events_time(graph.replay, args.steps, args.warmup, torch)

    def loop():
        for p, F, X in zip(plans, Fs, Xs):
            p.solve(F, "fp32_refined", out=X)
    ms_loop = _events_time(loop, max(3, min(args.steps, 10)), 2, torch)
    other = {}
    for strategy in ("per_series", "by_width", "grouped"):   # context: each layout of the same work
        tdm.set_batched_strategy(strategy)
        try:
            other[strategy] = _events_time(lambda: tdm.solve_batched(plans, Fs, "fp32_refined", outs=Xs),
                                           max(3, min(args.steps, 10)), 3, torch)
        finally:
            tdm.set_batched_strategy("auto")
    hbm, peak_kind = _peaks()
    achieved = unknowns * 12 / (ms_batched * 1e-3) / 1e9
    steps_used = sorted({p.info()["refine_steps"] for p in plans})
    line = {
        "metric": "unknowns solved/s, batched series (FP32 + refine to 1e-11)", "value": unknowns / (ms_batched * 1e-3),
        "unit": UNIT, "n_gpus": DIST["world"], "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batched,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batching: 512 Fourier-mode matrices (K=512), n ~ lognormal(2048) in [256, 65536], "
                               "N ~ U{1..2048}, F ~ N(0,1) fp32 drawn on the device, refined",
                   "matrices": len(specs), "unknowns": unknowns, "refine_steps": steps_used},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "peak_source": peak_kind, "kernel": "k_refined"},
        "paths": {"default_ms": ms_batched, "graph_replay_ms": ms_graph, "per_series_streams_ms": other["per_series"],
                  "by_width_ms": other["by_width"], "grouped_units_ms": other["grouped"],
                  "per_matrix_loop_ms": ms_loop, "speedup_vs_loop": ms_loop / ms_batched},
        "prepare_s_all_matrices": prepare_s,
    }
    for p in plans:
        p.close()
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)


def run_poisson(args):
    """The Fourier method of Section 4a on the paper's 1024 x 1024 mesh: a series
    of 100 model problems (eq. poisson_test) solved together: sine transforms,
    1023 mode series through the batched dichotomy solve, synthesis."""
    import numpy as np
    import torch
    from paper_0901_2859_gb300.poisson import FourierPoisson

    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    N1 = N2 = 1024
    nprob = 100
    t0 = time.perf_counter()
    fp = FourierPoisson(N1, N2, precision="fp32_refined", device=dev)
    torch.cuda.synchronize()
    prepare_s = time.perf_counter() - t0
    # the model right-hand side scaled per problem, so that every member of the series differs
    scale = torch.linspace(1.0, 2.0, nprob, dtype=torch.float64, device=dev)
    f = FourierPoisson.model_rhs(N1, N2, device=dev)[:, :, None] * scale
    steps = max(1, min(args.steps, 10))
    ms = _events_time(lambda: fp.solve(f), steps, max(3, args.warmup), torch)
    # error against the exact discrete solution of every problem
    h = 1.0 / N1
    lam = 8.0 / h ** 2 * np.sin(np.pi * h) ** 2
    ev = []
    u = fp.solve(f, events=ev)
    torch.cuda.synchronize()
    stages = {"analysis_ms": ev[0].elapsed_time(ev[1]), "mode_solves_ms": ev[1].elapsed_time(ev[2]),
              "synthesis_ms": ev[2].elapsed_time(ev[3])}
    err = float((u - f / lam).abs().max() / (f / lam).abs().max())
    fp.close()
    cpu = None
    if not args.no_cpu_baseline and DIST["rank"] == 0:
        # the oracle (explicit sine sums + binary64 sweeps) on one problem of the series
        import oracle
        from oracle import poisson as oracle_poisson
        f1 = f[:, :, 0].cpu().numpy()
        t0 = time.perf_counter()
        oracle_poisson.fourier_poisson(f1, 1.0 / N1, 1.0 / N2)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "problems/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"1 of the {nprob} problems, {dt:.1f} s"}
    line = {
        "metric": "Poisson problems solved/s (Fourier method, series of 100)", "value": nprob / (ms * 1e-3),
        "unit": "problems/s", "n_gpus": DIST["world"], "steps": steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "poisson2d: eq. poisson_test on a 1024 x 1024 mesh, 100 right-hand sides, "
                               "binary64 f split into two binary32 parts, refined dichotomy per mode",
                   "mesh": [N1, N2], "problems": nprob, "modes": N2 - 1},
        "rel_err_vs_exact_discrete": err,
        "stages": stages,
        "cpu_baseline": cpu,
        "prepare_s_all_modes": prepare_s,
        "paper_context": "833 problems/s on 1024 x 1024 (MBC-100k, best processor count; Section 5)",
    }
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)


def run_adi(args):
    """Alternating directions (Section 4b) on the paper's 1024 x 1024 mesh: a
    series of 100 model problems iterated together to eps = 1e-5 (binary64
    state, binary32 right-hand sides solved to binary64 results); the binary32
    variant is timed beside it."""
    import numpy as np
    import torch
    from paper_0901_2859_gb300.adi import PeacemanRachford
    from paper_0901_2859_gb300.poisson import FourierPoisson

    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    N, nprob, eps = 1024, 100, 1e-5
    t0 = time.perf_counter()
    pr = PeacemanRachford(N, eps, precision="fp32_refined", device=dev)
    torch.cuda.synchronize()
    prepare_s = time.perf_counter() - t0
    scale = torch.linspace(1.0, 2.0, nprob, dtype=torch.float64, device=dev)
    f = FourierPoisson.model_rhs(N, N, device=dev)[:, :, None] * scale
    steps = max(1, min(args.steps, 10))
    ms = _events_time(lambda: pr.solve(f), steps, max(3, args.warmup), torch)
    h = 1.0 / N
    lam = 8.0 / h ** 2 * np.sin(np.pi * h) ** 2
    u = pr.solve(f).double()
    err = float((u - f / lam).abs().max() / (f / lam).abs().max())
    iters = len(pr.omegas)
    # one half step's right-hand side alone (tdm_adi_rhs), along i and along j (transposed
    # views): binary64 v and f read, binary32 r written, 20 bytes per element
    n = N - 1
    buf = torch.empty((n, (n * nprob + 3) // 4 * 4), dtype=torch.float32, device=dev)
    om = float(pr.omegas[0])
    rhs_ms = [_events_time(lambda: pr._rhs(x, y, om, buf), steps, 3, torch)
              for x, y in ((u, f), (u.transpose(0, 1), f.transpose(0, 1)))]
    rhs_bytes = n * n * nprob * 20
    pr.close()
    pr32 = PeacemanRachford(N, eps, precision="fp32", device=dev)
    ms32 = _events_time(lambda: pr32.solve(f), steps, max(3, args.warmup), torch)
    u32 = pr32.solve(f).double()
    err32 = float((u32 - f / lam).abs().max() / (f / lam).abs().max())
    pr32.close()
    line = {
        "metric": "Poisson problems solved/s (alternating directions to eps = 1e-5, series of 100)",
        "value": nprob / (ms * 1e-3), "unit": "problems/s", "n_gpus": DIST["world"], "steps": steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adi: eq. poisson_test on a 1024 x 1024 mesh, 100 right-hand sides, Peaceman-Rachford "
                               "with n0(eps) geometric parameters, refined dichotomy solves (binary64 results)",
                   "mesh": [N, N], "problems": nprob, "iterations": iters, "eps": eps},
        "rel_err_vs_exact_discrete": err,
        "binary32_path": {"ms": ms32, "problems_per_s": nprob / (ms32 * 1e-3), "rel_err_vs_exact_discrete": err32},
        "rhs_kernel": {"ms_along_i": rhs_ms[0], "ms_along_j": rhs_ms[1], "bytes": rhs_bytes,
                       "gbs_along_i": rhs_bytes / (rhs_ms[0] * 1e6), "gbs_along_j": rhs_bytes / (rhs_ms[1] * 1e6)},
        "prepare_s_all_parameters": prepare_s,
        "paper_context": "about 30 problems/s on 1024 x 1024 (MBC-100k, best processor count; Table 2)",
    }
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)


def run_large(args):
    """A series beyond one cluster (n = 262144, N = 1024): the two-level solve,
    in every precision, with sampled columns checked against the oracle."""
    import numpy as np
    import torch
    import oracle
    import paper_0901_2859_gb300 as tdm

    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    n, N, s_shift = 262144, 1024, 1e-6
    a = -np.ones(n - 1)
    b = np.full(n, 2.0 + s_shift)
    rng = np.random.default_rng(DIST["rank"])
    F32 = torch.from_numpy(rng.standard_normal((n, N), dtype=np.float32)).to(dev)
    t0 = time.perf_counter()
    plan = tdm.prepare(a, b, device=dev)
    torch.cuda.synchronize()
    prepare_s = time.perf_counter() - t0
    paths = {}
    cols = np.array([0, 1, N // 2, N - 1])
    for prec, Fin, dt_out, bytes_per in (("fp32_refined", F32, torch.float64, 12), ("fp64", F32.double(), torch.float64, 16),
                                         ("fp32", F32, torch.float32, 8)):
        X = torch.empty((n, N), dtype=dt_out, device=dev)
        steps = max(3, min(args.steps, 20))
        ms = _events_time(lambda: plan.solve(Fin, prec, out=X), steps, args.warmup, torch)
        ref = oracle.solve_hi(a, b, Fin[:, cols].double().cpu().numpy())
        err = float(np.max(np.abs(X[:, cols].double().cpu().numpy() - ref)) / np.max(np.abs(ref)))
        hbm, _ = _peaks()
        paths[prec] = {"ms": ms, "unknowns_per_s": n * N / (ms * 1e-3), "rel_err_sampled": err,
                       "hbm_frac_algorithmic": n * N * bytes_per / (ms * 1e-3) / 1e9 / hbm}
        del X
    info = plan.info()
    plan.close()
    line = {
        "metric": "unknowns solved/s beyond one cluster (two-level solve)", "value": paths["fp32_refined"]["unknowns_per_s"],
        "unit": UNIT, "n_gpus": DIST["world"], "steps": max(3, min(args.steps, 20)), "warmup": args.warmup,
        "ms_per_step": paths["fp32_refined"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"large: n={n} N={N} s={s_shift} (a=-1, b=2+s), F~N(0,1) fp32; segments of 32768 rows",
                   "n": n, "N": N, "refine_steps": info["refine_steps"]},
        "paths": paths, "prepare_s": prepare_s,
    }
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)


def run_backward(args):
    """The backward of the solve (row A8) on the differentiation workload (n = 8192,
    N = 2048, a random dominant matrix): dF = A^{-1} W by the adjoint solve with
    the same plan (Lemma 2) and the deterministic row reductions of da, db, in the
    binary32 and the refined precision."""
    import torch
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads

    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    w = workloads.diff(seed=DIST["rank"])
    n, N = w.n, w.F.shape[1]
    plan = tdm.prepare(w.a, w.b, device=dev)
    F = torch.from_numpy(w.F).to(dev)
    W = torch.from_numpy(w.W).to(dev)
    hbm, peak_kind = _peaks()
    paths = {}
    # bytes per unknown: W read and dF written by the adjoint solve, dF and X read by the reductions
    for prec, x_dtype, w_in, bytes_per in (("fp32", torch.float32, W, 16), ("fp32_refined", torch.float64, W, 24)):
        X = plan.solve(F, prec)
        steps = max(3, min(args.steps, 20))
        ms = _events_time(lambda: plan.solve_backward(w_in, X, prec), steps, args.warmup, torch)
        paths[prec] = {"ms": ms, "unknowns_per_s": n * N / (ms * 1e-3), "bytes_per_unknown": bytes_per,
                       "hbm_frac": n * N * bytes_per / (ms * 1e-3) / 1e9 / hbm}
        del X
    plan.close()
    line = {
        "metric": "unknowns/s of the backward (dF, da, db)", "value": paths["fp32"]["unknowns_per_s"], "unit": UNIT,
        "n_gpus": DIST["world"], "steps": max(3, min(args.steps, 20)), "warmup": args.warmup,
        "ms_per_step": paths["fp32"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"backward: diff n={n} N={N}, a ~ U[-1,-0.5], b ~ U[2.2,3], F, W ~ N(0,1) fp32",
                   "n": n, "N": N},
        "roofline": {"bound": "hbm", "achieved": n * N * 16 / (paths["fp32"]["ms"] * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": paths["fp32"]["hbm_frac"], "traffic": None, "peak_source": peak_kind,
                     "kernel": "k_solve<float> + k_grad_rows"},
        "paths": paths,
    }
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)


def run_algorithm2(args):
    """Algorithm 2 (Section 3.1) at the benchmark size: every separator value of
    the precision series (P = M - 1 = 511 components) as G^T F, by the library's
    tensor-core kernel (three TF32 products, tcgen05) and in binary64; the
    dichotomy's own separator values are the reference.  For context, the same
    three TF32 products as cuBLAS GEMMs."""
    import numpy as np
    import torch
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    from paper_0901_2859_gb300.algorithm2 import _tf32_split, components, inverse_rows

    dev = torch.device("cuda", DIST["local"])
    torch.cuda.set_device(dev)
    n, N = N_ROWS, 8192
    s = workloads.precision(seed=0, n=n, N=N, s=SHIFT)
    plan = tdm.prepare(s.a, s.b, device=dev)
    t = plan.info()["block_rows"]
    ks = list(range(t, n, t))                      # the separator rows
    F = torch.from_numpy(s.F).to(dev)
    ref = plan.solve(F.double(), "fp64")[ks]
    steps = max(3, min(args.steps, 10))
    G = inverse_rows(plan, ks)
    ms_g = _events_time(lambda: inverse_rows(plan, ks), steps, 3, torch)

    def cublas_tf32x3():   # context only: library GEMMs on the same split operands
        gh, gt = _tf32_split(G.t().to(torch.float32).contiguous())
        fh, ft = _tf32_split(F)
        X = torch.matmul(gh, fh)
        X += torch.matmul(gh, ft)
        X += torch.matmul(gt, fh)
        return X

    out = {}
    for mode, fn, k in (("tc", lambda: components(plan, F, ks, "tc", G=G), steps),
                        ("fp64", lambda: components(plan, F, ks, "fp64", G=G), 3),
                        ("cublas_tf32x3", cublas_tf32x3, steps)):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = mode == "cublas_tf32x3"
        try:
            ms = _events_time(fn, k, 3, torch)
            X = fn().double()
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
        err = float(((X - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)).max())
        flops = 2.0 * len(ks) * n * N * (1 if mode == "fp64" else 3)
        out[mode] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12, "rel_err_vs_dichotomy": err}
    plan.close()
    line = {
        "metric": "separator values by Algorithm 2 (dense G^T F)", "value": out["tc"]["ms"], "unit": "ms",
        "n_gpus": DIST["world"], "steps": steps, "warmup": 3, "ms_per_step": out["tc"]["ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3", "data": "synthetic",
        "config": {"workload": f"algorithm2: precision series n={n} N={N}, {len(ks)} separator components",
                   "components": len(ks), "kernel": "k_alg2_tc (tcgen05.mma kind::tf32, split-K 1024)"},
        "paths": out, "inverse_rows_ms": ms_g,
    }
    if DIST["rank"] == 0:
        print(json.dumps(line), flush=True)


def run_reference(args):
    """The oracle (the plain CPU implementation), timed on the host cores on a bounded sample."""
    N_RHS = args.rhs
    if DIST["rank"] != 0:
        return
    import numpy as np
    import oracle
    from paper_0901_2859_gb300 import workloads
    oracle.build()
    series = workloads.precision(seed=0, n=N_ROWS, N=N_RHS, s=SHIFT)
    threads = oracle.max_threads()
    probe = np.ascontiguousarray(series.F[:, :256], dtype=np.float64)
    t0 = time.perf_counter()
    oracle.thomas_f64(series.a, series.b, probe, threads=threads)
    per_col = (time.perf_counter() - t0) / 256
    budget = 90.0 / max(1, args.steps + args.warmup)          # seconds per step
    k = int(max(16, min(N_RHS, budget / max(per_col, 1e-9))))
    Fs = np.ascontiguousarray(series.F[:, :k], dtype=np.float64)
    for _ in range(args.warmup):
        oracle.thomas_f64(series.a, series.b, Fs, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.thomas_f64(series.a, series.b, Fs, threads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    value = N_ROWS * k / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": DIST["world"],
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_ROWS, "N": N_RHS, "s": SHIFT},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"oracle binary64 sweep (thomas_f64) on {k} of {N_RHS} right-hand sides per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-cols", type=int, default=8192, help="columns of the CPU baseline sample")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU baseline: seconds of repeated passes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="precision", choices=["precision", "batching", "poisson2d", "adi", "large", "algorithm2", "backward"],
                    help="precision: the benchmark line; batching: 512 matrices of uneven size in one call; "
                         "poisson2d: the Fourier method on a 1024 x 1024 mesh, 100 problems; adi: alternating directions; "
                         "large: the two-level solve beyond one cluster; algorithm2: separator values as dense products; "
                         "backward: the gradient of the solve")
    ap.add_argument("--rhs", type=int, default=N_RHS,
                    help="right-hand sides of the series (the benchmark is 8192; smaller values are for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "algorithm2":
        run_algorithm2(args)
    elif args.workload == "backward":
        run_backward(args)
    elif args.workload == "large":
        run_large(args)
    elif args.workload == "adi":
        run_adi(args)
    elif args.workload == "poisson2d":
        run_poisson(args)
    elif args.workload == "batching":
        run_batching(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
