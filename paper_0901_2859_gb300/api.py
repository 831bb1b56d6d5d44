"""Python binding of the tdm C ABI: argument marshalling over torch tensors.

Every step of the solve runs in the CUDA library; this module only checks
dtypes, devices and strides, passes raw device pointers and the current CUDA
stream, and turns status codes into exceptions.  There is no CPU fallback: a
missing library or a non-CUDA tensor raises.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import PRECISIONS, TDMError, TDMInfo, TDMOptions, check

__all__ = ["Plan", "prepare", "solve_batched", "solve_batched_noalloc", "TDMSolve", "tdm_solve", "TDMError"]

_OUT_DTYPE = {"fp64": torch.float64, "fp32": torch.float32, "fp32_refined": torch.float64}
_IN_DTYPE = {"fp64": torch.float64, "fp32": torch.float32, "fp32_refined": torch.float32}


def _stream_ptr(device: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_rhs(T: torch.Tensor, n: int, dtype: torch.dtype, name: str) -> int:
    if not isinstance(T, torch.Tensor) or not T.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if T.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {T.dtype}")
    if T.dim() != 2 or T.shape[0] != n:
        raise ValueError(f"{name} must have shape (n={n}, N), got {tuple(T.shape)}")
    if T.shape[1] > 0 and T.stride(1) != 1:
        raise ValueError(f"{name} must have unit stride along the right-hand sides")
    return max(int(T.stride(0)), int(T.shape[1]))


class Plan:
    """A prepared matrix (Algorithm 3/4 step 1).  Owns device memory until closed."""

    def __init__(self, a: torch.Tensor, b: torch.Tensor, block_rows: int = 0, refine_steps: int = 0,
                 tile_rhs: int = 0, sup: torch.Tensor | None = None):
        """A = tridiag(a, b, a); with `sup`, the nonsymmetric A with sub-diagonal a
        (A[k+1][k]) and super-diagonal sup (A[k][k+1]) (Section 3.5)."""
        lib = _lib.load()
        if not (isinstance(b, torch.Tensor) and b.is_cuda):
            raise TypeError("a and b must be CUDA tensors (float64)")
        n = int(b.shape[0])
        a = a.to(device=b.device, dtype=torch.float64).contiguous()
        b = b.to(dtype=torch.float64).contiguous()
        if a.numel() != max(n - 1, 0):
            raise ValueError(f"a must have n-1 = {n - 1} entries, got {a.numel()}")
        if sup is not None:
            sup = sup.to(device=b.device, dtype=torch.float64).contiguous()
            if sup.numel() != max(n - 1, 0):
                raise ValueError(f"sup must have n-1 = {n - 1} entries, got {sup.numel()}")
        self.device = b.device
        self.n = n
        self.general = sup is not None
        opts = TDMOptions(block_rows, refine_steps, 0, tile_rhs)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if self.general:
                st = lib.tdm_prepare_general(ctypes.c_void_p(a.data_ptr() if n > 1 else 0),
                                             ctypes.c_void_p(b.data_ptr()),
                                             ctypes.c_void_p(sup.data_ptr() if n > 1 else 0), n,
                                             ctypes.byref(opts), _stream_ptr(self.device), ctypes.byref(h))
            else:
                st = lib.tdm_prepare(ctypes.c_void_p(a.data_ptr() if n > 1 else 0), ctypes.c_void_p(b.data_ptr()),
                                     n, ctypes.byref(opts), _stream_ptr(self.device), ctypes.byref(h))
        check(st, "tdm_prepare_general" if self.general else "tdm_prepare")
        self._h = h
        self.a, self.b = a, b   # kept for autograd and the residual-free properties
        self.sup = sup

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    def info(self) -> dict:
        inf = TDMInfo()
        check(_lib.load().tdm_get_info(self.handle, ctypes.byref(inf)), "tdm_get_info")
        return {f: getattr(inf, f) for f, _ in TDMInfo._fields_}

    def solve(self, F: torch.Tensor, precision: str = "fp32", out: torch.Tensor | None = None) -> torch.Tensor:
        """X = A^{-1} F for every column of F (shape (n, N), right-hand sides contiguous)."""
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {list(PRECISIONS)}")
        ldF = _check_rhs(F, self.n, _IN_DTYPE[precision], "F")
        N = int(F.shape[1])
        if out is None:
            out = torch.empty((self.n, N), dtype=_OUT_DTYPE[precision], device=F.device)
        ldX = _check_rhs(out, self.n, _OUT_DTYPE[precision], "out")
        if out.shape[1] != N:
            raise ValueError("out must have as many columns as F")
        with torch.cuda.device(self.device):
            st = _lib.load().tdm_solve(self.handle, ctypes.c_void_p(F.data_ptr()), ldF,
                                       ctypes.c_void_p(out.data_ptr()), ldX, N, PRECISIONS[precision],
                                       _stream_ptr(self.device))
        check(st, "tdm_solve")
        return out

    def solve_host(self, F: torch.Tensor, precision: str = "fp32", out: torch.Tensor | None = None,
                   chunk: int = 0) -> torch.Tensor:
        """X = A^{-1} F for F and X in host memory (pin them for overlapped copies):
        ``tdm_solve_host`` copies chunks of columns in, solves and copies them out on
        separate streams.  Enqueued on the current stream; synchronize before reading X."""
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {list(PRECISIONS)}")
        if not isinstance(F, torch.Tensor) or F.is_cuda:
            raise TypeError("F must be a host (CPU) tensor")
        if F.dtype != _IN_DTYPE[precision] or F.dim() != 2 or F.shape[0] != self.n or (F.shape[1] and F.stride(1) != 1):
            raise ValueError(f"F must be a ({self.n}, N) {_IN_DTYPE[precision]} host tensor with unit column stride")
        N = int(F.shape[1])
        if out is None:
            out = torch.empty((self.n, N), dtype=_OUT_DTYPE[precision], pin_memory=F.is_pinned())
        if out.is_cuda or out.dtype != _OUT_DTYPE[precision] or tuple(out.shape) != (self.n, N) or \
                (N and out.stride(1) != 1):
            raise ValueError(f"out must be a ({self.n}, {N}) {_OUT_DTYPE[precision]} host tensor with unit column stride")
        ldF, ldX = max(int(F.stride(0)), N), max(int(out.stride(0)), N)
        with torch.cuda.device(self.device):
            st = _lib.load().tdm_solve_host(self.handle, ctypes.c_void_p(F.data_ptr()), ldF,
                                            ctypes.c_void_p(out.data_ptr()), ldX, N, int(chunk),
                                            PRECISIONS[precision], _stream_ptr(self.device))
        check(st, "tdm_solve_host")
        return out

    def solve_backward(self, W: torch.Tensor, X: torch.Tensor, precision: str = "fp32",
                       need_ab: bool = True):
        """(dF, da, db) for L with dL/dX = W, X = A^{-1} F (adjoint solve, Lemma 2)."""
        ld = _check_rhs(W, self.n, _IN_DTYPE[precision], "W")
        ldx = _check_rhs(X, self.n, _OUT_DTYPE[precision], "X")
        N = int(W.shape[1])
        if ld != ldx:
            W, X = W.contiguous(), X.contiguous()
            ld = max(N, 1)
        dF = torch.empty_strided((self.n, N), (ld, 1), dtype=_OUT_DTYPE[precision], device=W.device)
        da = torch.empty(max(self.n - 1, 0), dtype=torch.float64, device=W.device) if need_ab else None
        db = torch.empty(self.n, dtype=torch.float64, device=W.device) if need_ab else None
        with torch.cuda.device(self.device):
            st = _lib.load().tdm_solve_backward(
                self.handle, ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(X.data_ptr()), ld, N,
                ctypes.c_void_p(dF.data_ptr()),
                ctypes.c_void_p(da.data_ptr() if (da is not None and da.numel()) else 0),
                ctypes.c_void_p(db.data_ptr() if db is not None else 0),
                PRECISIONS[precision], _stream_ptr(self.device))
        check(st, "tdm_solve_backward")
        return dF, da, db

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib.load().tdm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def prepare_general(sub, diag, sup, block_rows: int = 0, device=None) -> Plan:
    """Prepare a nonsymmetric tridiagonal A (A[k+1][k] = sub[k], A[k][k] = diag[k],
    A[k][k+1] = sup[k]) with every sub[k] * sup[k] > 0: symmetrized by the
    diagonal similarity of Section 3.5.  The plan serves "fp64" and "fp32" solves."""
    dev = torch.device(device) if device is not None else (
        diag.device if isinstance(diag, torch.Tensor) and diag.is_cuda else torch.device("cuda", torch.cuda.current_device()))
    as_dev = lambda x: torch.as_tensor(x, dtype=torch.float64).to(dev)
    return Plan(as_dev(sub), as_dev(diag), block_rows=block_rows, sup=as_dev(sup))


def prepare(a, b, block_rows: int = 0, refine_steps: int = 0, device=None, tile_rhs: int = 0) -> Plan:
    """Prepare A = tridiag(a, b, a); a, b may be CUDA tensors or host arrays."""
    if not isinstance(b, torch.Tensor) or not b.is_cuda:
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        b = torch.as_tensor(b, dtype=torch.float64).to(dev)
        a = torch.as_tensor(a, dtype=torch.float64).to(dev)
    return Plan(a, b, block_rows=block_rows, refine_steps=refine_steps, tile_rhs=tile_rhs)


BATCHED_STRATEGIES = {"by_width": 0, "grouped": 1, "per_series": 2, "auto": 3, "cooperative": 4}


def set_batched_strategy(strategy: str) -> None:
    """How ``solve_batched`` lays out refined work (``tdm_set_batched_strategy``):
    "auto" (default) -- "by_width" for batches needing at most four launch
    classes, else "per_series"; "per_series" -- one single-series launch per
    series over four streams; "by_width" -- one persistent launch per kernel
    shape and cluster width; "grouped" -- one per kernel shape, tiles of
    several series side by side in each cluster."""
    check(_lib.load().tdm_set_batched_strategy(BATCHED_STRATEGIES[strategy]), "tdm_set_batched_strategy")


def solve_batched(plans, Fs, precision: str = "fp32_refined", outs=None):
    """Solve every plans[k] against Fs[k] in one call (persistent launches over
    a device-resident work list; see ``set_batched_strategy``)."""
    if len(plans) != len(Fs):
        raise ValueError("plans and Fs must have the same length")
    count = len(plans)
    if outs is None:
        outs = [torch.empty((p.n, F.shape[1]), dtype=_OUT_DTYPE[precision], device=F.device)
                for p, F in zip(plans, Fs)]
    hs = (ctypes.c_void_p * count)(*[p.handle.value for p in plans])
    fp = (ctypes.c_void_p * count)()
    xp = (ctypes.c_void_p * count)()
    ldf = (ctypes.c_int64 * count)()
    ldx = (ctypes.c_int64 * count)()
    ns = (ctypes.c_int64 * count)()
    for k, (p, F, X) in enumerate(zip(plans, Fs, outs)):
        ldf[k] = _check_rhs(F, p.n, _IN_DTYPE[precision], f"Fs[{k}]")
        ldx[k] = _check_rhs(X, p.n, _OUT_DTYPE[precision], f"outs[{k}]")
        fp[k] = F.data_ptr()
        xp[k] = X.data_ptr()
        ns[k] = int(F.shape[1])
    dev = plans[0].device if count else torch.device("cuda")
    with torch.cuda.device(dev):
        st = _lib.load().tdm_solve_batched(hs, count, fp, ldf, xp, ldx, ns, PRECISIONS[precision],
                                           _stream_ptr(dev))
    check(st, "tdm_solve_batched")
    return outs


def solve_batched_noalloc(plans, Fs, outs):
    """``solve_batched`` (refined) through ``tdm_solve_batched_noalloc``: the
    library allocates nothing; the caller provides every output."""
    if not (len(plans) == len(Fs) == len(outs)):
        raise ValueError("plans, Fs and outs must have the same length")
    count = len(plans)
    hs = (ctypes.c_void_p * count)(*[p.handle.value for p in plans])
    fp = (ctypes.c_void_p * count)()
    xp = (ctypes.c_void_p * count)()
    ldf = (ctypes.c_int64 * count)()
    ldx = (ctypes.c_int64 * count)()
    ns = (ctypes.c_int64 * count)()
    for k, (p, F, X) in enumerate(zip(plans, Fs, outs)):
        ldf[k] = _check_rhs(F, p.n, torch.float32, f"Fs[{k}]")
        ldx[k] = _check_rhs(X, p.n, torch.float64, f"outs[{k}]")
        fp[k] = F.data_ptr()
        xp[k] = X.data_ptr()
        ns[k] = int(F.shape[1])
    dev = plans[0].device if count else torch.device("cuda")
    with torch.cuda.device(dev):
        st = _lib.load().tdm_solve_batched_noalloc(hs, count, fp, ldf, xp, ldx, ns, _stream_ptr(dev))
    check(st, "tdm_solve_batched_noalloc")
    return outs


class TDMSolve(torch.autograd.Function):
    """X = A^{-1} F with gradients for F, a and b through the adjoint solve."""

    @staticmethod
    def forward(ctx, F, a, b, plan: Plan, precision: str = "fp32"):
        X = plan.solve(F.contiguous(), precision=precision)
        ctx.plan, ctx.precision = plan, precision
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        need_ab = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        # W takes the forward input's dtype (binary32 for the refined solve, whose X is binary64)
        dF, da, db = ctx.plan.solve_backward(gX.contiguous().to(_IN_DTYPE[ctx.precision]), X, ctx.precision,
                                             need_ab=need_ab)
        dF = dF.to(_IN_DTYPE[ctx.precision])
        da = da.to(ctx.plan.a.dtype) if (da is not None and ctx.needs_input_grad[1]) else None
        db = db.to(ctx.plan.b.dtype) if (db is not None and ctx.needs_input_grad[2]) else None
        return dF, da, db, None, None


def tdm_solve(F, a, b, plan: Plan, precision: str = "fp32"):
    return TDMSolve.apply(F, a, b, plan, precision)
