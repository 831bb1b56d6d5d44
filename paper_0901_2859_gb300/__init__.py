"""GB300-native parallel dichotomy solver for series of symmetric tridiagonal systems.

A. V. Terekhov, "Parallel dichotomy algorithm for solving tridiagonal SLAEs":
a once-per-matrix preparation (inverse rows at block separators, homogeneous
ratios, local sweep coefficients) and a per-right-hand-side solve (block dot
products, separator values by the main parallel sweep theorem, local sweeps
with a correction), all as CUDA kernels for sm_103a behind the C ABI in
``include/tdm.h``.  This package is the thin Python binding over that ABI.
"""
from .api import Plan, TDMError, TDMSolve, prepare, prepare_general, set_batched_strategy, solve_batched, solve_batched_noalloc, tdm_solve  # noqa: F401
from ._build import build  # noqa: F401
from . import autotune  # noqa: F401

__all__ = ["Plan", "TDMError", "TDMSolve", "prepare", "prepare_general", "set_batched_strategy", "solve_batched", "solve_batched_noalloc", "tdm_solve", "build"]
