"""Algorithm 2 of Section 3.1: selected solution components as dense products.

For components k_1..k_P of every solution X_n of the series A X_n = F_n:

  1. G_k solves A G_k = e_k (Lemma 2: the k-th row of A^-1), once for the
     series: P unit right-hand sides through the plan's own dichotomy solve;
  2. X[k, :] = G_k^T F for all right-hand sides at once: one (P x n)(n x N)
     matrix product.

The product:

* ``"tc"`` (the default): the library's tensor-core kernel (``tdm_algorithm2``,
  tcgen05.mma on TF32 operands, binary32 accumulation in tensor memory), as
  three TF32 products of the heads and tails of G and F, each binary32
  accumulation over at most 1024 rows of K, the partial sums added in binary32
  pairs; binary32 result;
* ``"fp64"``: a binary64 library GEMM (``torch.matmul``), the reference.

Algorithm 2 is the theorem-free route to the separator values: it checks the
dichotomy's Theorem 2 path independently, and it serves a caller who needs a
few components of a long series.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check
from .api import Plan

__all__ = ["inverse_rows", "components"]


def inverse_rows(plan: Plan, ks) -> torch.Tensor:
    """G = [G_k1 .. G_kP], shape (n, P), binary64: A G = [e_k1 .. e_kP]."""
    ks = torch.as_tensor(ks, dtype=torch.int64, device=plan.device).reshape(-1)
    if ks.numel() and (int(ks.min()) < 0 or int(ks.max()) >= plan.n):
        raise ValueError("component index out of range")
    P = int(ks.numel())
    ld = max(2, (P + 1) // 2 * 2)   # a 16-byte row pitch
    E = torch.zeros((plan.n, ld), dtype=torch.float64, device=plan.device)
    E[ks, torch.arange(P, device=plan.device)] = 1.0
    G = torch.empty_like(E)
    plan.solve(E[:, :P], "fp64", out=G[:, :P])
    return G[:, :P]


def _tf32_split(x: torch.Tensor):
    """x (binary32) = head + tail, the head's significand cut to TF32's 10 bits
    (the split the tensor-core kernel applies to F and G)."""
    head = (x.view(torch.int32) & torch.tensor(-8192, dtype=torch.int32, device=x.device)).view(torch.float32)
    return head, x - head


def components(plan: Plan, F: torch.Tensor, ks, mode: str = "tc", G: torch.Tensor | None = None) -> torch.Tensor:
    """X[k, :] for the components ks of the solutions of A X = F (F shape (n, N));
    returns (P, N): binary32 for "tc", binary64 for "fp64".  Pass G from
    inverse_rows to reuse it across calls."""
    if mode not in ("fp64", "tc"):
        raise ValueError("mode must be 'tc' or 'fp64'")
    if F.dim() != 2 or F.shape[0] != plan.n:
        raise ValueError(f"F must have shape ({plan.n}, N)")
    if G is None:
        G = inverse_rows(plan, ks)
    if mode == "fp64":
        return G.t() @ F.to(torch.float64)
    P, n, N = int(G.shape[1]), plan.n, int(F.shape[1])
    F32 = F.to(torch.float32)
    if F32.stride(1) != 1 or F32.stride(0) % 4 or F32.data_ptr() % 16:   # the copy engine's alignment
        pad = torch.empty((n, (N + 3) // 4 * 4), dtype=torch.float32, device=F.device)
        pad[:, :N] = F32
        F32 = pad
    X = torch.empty((P, max(N, 1)), dtype=torch.float32, device=F.device)[:, :N]
    lib = _lib.load()
    nbytes = lib.tdm_algorithm2_workspace(min(P, 512), n, N)
    work = torch.empty(nbytes, dtype=torch.uint8, device=F.device)
    with torch.cuda.device(F.device):
        st = lib.tdm_algorithm2(ctypes.c_void_p(G.data_ptr()), int(G.stride(0)), P, n,
                                ctypes.c_void_p(F32.data_ptr()), int(F32.stride(0)), N,
                                ctypes.c_void_p(X.data_ptr()), int(X.stride(0)) if N else 1,
                                ctypes.c_void_p(work.data_ptr()), nbytes,
                                ctypes.c_void_p(torch.cuda.current_stream(F.device).cuda_stream))
    check(st, "tdm_algorithm2")
    return X
