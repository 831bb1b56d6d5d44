"""ctypes declarations of the C ABI in ``include/tdm.h`` (marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

TDM_OK = 0
STATUS_NAMES = {
    0: "TDM_OK", 1: "TDM_ERR_INVALID_ARG", 2: "TDM_ERR_SINGULAR", 3: "TDM_ERR_CUDA",
    4: "TDM_ERR_NO_MEMORY", 5: "TDM_ERR_NOT_CONVERGED", 6: "TDM_ERR_TIMEOUT",
    7: "TDM_ERR_NOT_IMPLEMENTED", 8: "TDM_ERR_TOO_LARGE",
}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_refined": 2}

# every symbol include/tdm.h declares
EXPORTS = ("tdm_prepare", "tdm_prepare_general", "tdm_solve", "tdm_solve_host", "tdm_solve_batched", "tdm_solve_batched_noalloc", "tdm_set_batched_strategy", "tdm_selftest_group_timeout", "tdm_adi_rhs",
           "tdm_solve_backward", "tdm_selftest_wait_timeout", "tdm_get_info", "tdm_destroy",
           "tdm_status_string", "tdm_algorithm2_workspace", "tdm_algorithm2", "tdm_algorithm2_status")
NOALLOC_MAX_TILES = 4096   # TDM_NOALLOC_MAX_TILES


class TDMOptions(ctypes.Structure):
    _fields_ = [("block_rows", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("flags", ctypes.c_int), ("tile_rhs", ctypes.c_int)]


class TDMInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("block_rows", ctypes.c_int32), ("num_blocks", ctypes.c_int32),
                ("dominant", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("max_abs_z", ctypes.c_double), ("min_abs_pivot", ctypes.c_double),
                ("device_error", ctypes.c_int32), ("tile_rhs", ctypes.c_int32), ("general", ctypes.c_int32),
                ("contraction", ctypes.c_float)]


class TDMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libtdm.so (building it first if it is missing).  Never falls back."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise OSError(f"{path} is missing; run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.tdm_prepare.argtypes = [vp, vp, i64, ctypes.POINTER(TDMOptions), vp, ctypes.POINTER(vp)]
        lib.tdm_prepare_general.argtypes = [vp, vp, vp, i64, ctypes.POINTER(TDMOptions), vp, ctypes.POINTER(vp)]
        lib.tdm_solve.argtypes = [vp, vp, i64, vp, i64, i64, i32, vp]
        lib.tdm_solve_host.argtypes = [vp, vp, i64, vp, i64, i64, i64, i32, vp]
        lib.tdm_solve_batched.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                          ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i64), i32, vp]
        lib.tdm_solve_batched_noalloc.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp),
                                                  ctypes.POINTER(i64), ctypes.POINTER(vp),
                                                  ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
        lib.tdm_solve_backward.argtypes = [vp, vp, vp, i64, i64, vp, vp, vp, i32, vp]
        lib.tdm_set_batched_strategy.argtypes = [i32]
        lib.tdm_get_info.argtypes = [vp, ctypes.POINTER(TDMInfo)]
        lib.tdm_selftest_wait_timeout.argtypes = [i64, vp]
        lib.tdm_selftest_group_timeout.argtypes = [i64, vp]
        lib.tdm_adi_rhs.argtypes = [vp, i64, i64, vp, i64, i64, i64, i64, i64, ctypes.c_double, ctypes.c_double,
                                    i32, vp, i64, i32, vp]
        lib.tdm_destroy.argtypes = [vp]
        lib.tdm_status_string.argtypes = [i32]
        lib.tdm_algorithm2_workspace.argtypes = [i64, i64, i64]
        lib.tdm_algorithm2.argtypes = [vp, i64, i64, i64, vp, i64, i64, vp, i64, vp, ctypes.c_size_t, vp]
        lib.tdm_algorithm2_status.argtypes = [vp, i64, i64, i64, vp, ctypes.POINTER(i32)]
        for name in EXPORTS:
            getattr(lib, name).restype = ctypes.c_int
        lib.tdm_status_string.restype = ctypes.c_char_p
        lib.tdm_algorithm2_workspace.restype = ctypes.c_size_t
        _lib = lib
        return lib


def check(status: int, what: str) -> None:
    if status != TDM_OK:
        raise TDMError(status, what)
