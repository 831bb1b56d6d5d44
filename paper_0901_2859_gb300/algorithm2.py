"""Algorithm 2 of Section 3.1: selected solution components as dense products.

For components k_1..k_P of every solution X_n of the series A X_n = F_n:

  1. G_k solves A G_k = e_k (Lemma 2: the k-th row of A^-1), once for the
     series: P unit right-hand sides through the plan's own dichotomy solve;
  2. X[k, :] = G_k^T F for all right-hand sides at once: one (P x n)(n x N)
     matrix product.

The product is a plain library GEMM (cuBLAS through ``torch.matmul``):

* ``"fp64"``: in binary64;
* ``"tf32x3"``: on the tensor cores, G and F each split into a TF32 head and
  a TF32 tail, with the three products that matter (head x head, head x tail,
  tail x head) accumulated in binary32; about binary32 accuracy at tensor-core
  rate.

Algorithm 2 is the theorem-free route to the separator values: it checks the
dichotomy's Theorem 2 path independently, and it serves a caller who needs a
few components of a long series.
"""
from __future__ import annotations

import torch

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
    """x (binary32) = head + tail, the head's significand cut to TF32's 10 bits."""
    head = (x.view(torch.int32) & torch.tensor(-8192, dtype=torch.int32, device=x.device)).view(torch.float32)
    return head, x - head


def components(plan: Plan, F: torch.Tensor, ks, mode: str = "fp64", G: torch.Tensor | None = None) -> torch.Tensor:
    """X[k, :] for the components ks of the solutions of A X = F (F shape (n, N));
    returns (P, N): binary64 for "fp64", binary32 for "tf32x3".  Pass G from
    inverse_rows to reuse it across calls."""
    if mode not in ("fp64", "tf32x3"):
        raise ValueError("mode must be 'fp64' or 'tf32x3'")
    if F.dim() != 2 or F.shape[0] != plan.n:
        raise ValueError(f"F must have shape ({plan.n}, N)")
    if G is None:
        G = inverse_rows(plan, ks)
    if mode == "fp64":
        return G.t() @ F.to(torch.float64)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        gh, gt = _tf32_split(G.t().to(torch.float32).contiguous())
        fh, ft = _tf32_split(F.to(torch.float32).contiguous())
        X = gh @ fh
        X += gh @ ft
        X += gt @ fh
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return X
