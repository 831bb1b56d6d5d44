"""The C-ABI library loads, exports every symbol include/tdm.h declares, and
rejects invalid arguments on the host (no GPU work is issued by these calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "tdm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_0901_2859_gb300 import _lib
    return _lib.load()


def test_header_declares_the_documented_entry_points():
    from paper_0901_2859_gb300 import _lib
    assert _declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_0901_2859_gb300 import _lib
    for code, name in _lib.STATUS_NAMES.items():
        assert lib.tdm_status_string(code).decode() == name
    assert lib.tdm_status_string(99).decode() == "TDM_ERR_UNKNOWN"


def test_host_validation_rejects_bad_arguments(lib):
    vp = ctypes.c_void_p
    h = vp()
    fake = vp(0x10000)
    # tdm_prepare: null out, n < 1, null b, misaligned b
    assert lib.tdm_prepare(fake, fake, 10, None, None, None) == 1
    assert lib.tdm_prepare(fake, fake, 0, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.tdm_prepare(fake, None, 10, None, None, ctypes.byref(h)) == 1
    assert lib.tdm_prepare(fake, vp(0x10004), 10, None, None, ctypes.byref(h)) == 1
    # tdm_solve / backward / info with a null handle
    assert lib.tdm_solve(None, fake, 4, vp(0x20000), 4, 4, 1, None) == 1
    assert lib.tdm_solve_backward(None, fake, fake, 4, 4, fake, None, None, 1, None) == 1
    assert lib.tdm_get_info(None, None) == 1
    # batched: negative count, null arrays
    assert lib.tdm_solve_batched(None, -1, None, None, None, None, None, 2, None) == 1
    assert lib.tdm_solve_batched(None, 3, None, None, None, None, None, 2, None) == 1
    assert lib.tdm_solve_batched(None, 0, None, None, None, None, None, 2, None) == 0
    # batched without allocation: negative count, null arrays, empty call
    assert lib.tdm_solve_batched_noalloc(None, -1, None, None, None, None, None, None) == 1
    assert lib.tdm_solve_batched_noalloc(None, 2, None, None, None, None, None, None) == 1
    assert lib.tdm_solve_batched_noalloc(None, 0, None, None, None, None, None, None) == 0
    # destroy(NULL) is accepted
    assert lib.tdm_destroy(None) == 0


def test_general_prepare_validation(lib):
    from paper_0901_2859_gb300._lib import TDMOptions
    h = ctypes.c_void_p()
    # null diagonal, null off-diagonals with n > 1, n out of range: rejected before any CUDA call
    assert lib.tdm_prepare_general(None, None, None, 10, None, None, ctypes.byref(h)) == 1
    assert lib.tdm_prepare_general(None, ctypes.c_void_p(0x20000), ctypes.c_void_p(0x30000), 10, None, None,
                                   ctypes.byref(h)) == 1
    assert lib.tdm_prepare_general(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), ctypes.c_void_p(0x30000), 0,
                                   None, None, ctypes.byref(h)) == 1
    assert lib.tdm_prepare_general(ctypes.c_void_p(0x10004), ctypes.c_void_p(0x20000), ctypes.c_void_p(0x30000), 10,
                                   None, None, ctypes.byref(h)) == 1   # misaligned
    opt = TDMOptions(24, 0, 0, 0)
    assert lib.tdm_prepare_general(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), ctypes.c_void_p(0x30000), 10,
                                   ctypes.byref(opt), None, ctypes.byref(h)) == 1
    assert h.value is None


def test_bad_block_rows_rejected_before_any_cuda_call(lib):
    from paper_0901_2859_gb300._lib import TDMOptions
    h = ctypes.c_void_p()
    opt = TDMOptions(24, 0, 0, 0)
    assert lib.tdm_prepare(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 100, ctypes.byref(opt),
                           None, ctypes.byref(h)) == 1
    opt = TDMOptions(32, 0, 0, 5)            # tile_rhs must be 0, 4, 8 or 16
    assert lib.tdm_prepare(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 100, ctypes.byref(opt),
                           None, ctypes.byref(h)) == 1
    opt = TDMOptions(32, -2, 0, 0)
    assert lib.tdm_prepare(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 100, ctypes.byref(opt),
                           None, ctypes.byref(h)) == 1
    opt = TDMOptions(32, 9, 0, 0)
    assert lib.tdm_prepare(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 100, ctypes.byref(opt),
                           None, ctypes.byref(h)) == 1


def test_host_solve_validation(lib):
    # rejected before any CUDA call: null handle, negative chunk, N < 0, bad precision
    assert lib.tdm_solve_host(None, ctypes.c_void_p(0x1000), 4, ctypes.c_void_p(0x9000), 4, 4, 0, 2, None) == 1


def test_adi_rhs_validation(lib):
    # rejected (or, when empty, accepted) before any CUDA call
    vp, fake, d = ctypes.c_void_p, ctypes.c_void_p(0x10000), ctypes.c_double
    def call(v, f, R, na, nb, S, ldR, in64, out64):
        return lib.tdm_adi_rhs(v, nb * S, S, f, nb * S, S, na, nb, S, d(-2.0), d(1.0), in64, R, ldR, out64, None)
    assert call(fake, fake, fake, -1, 4, 2, 8, 1, 1) == 1
    assert call(fake, fake, fake, 4, 4, -2, 8, 1, 1) == 1
    assert call(fake, fake, fake, 4, 4, 2, 8, 0, 1) == 1        # binary32 in, binary64 out
    assert call(fake, fake, fake, 0, 4, 2, 8, 1, 1) == 0        # empty
    assert call(None, fake, fake, 4, 4, 2, 8, 1, 1) == 1
    assert call(fake, fake, None, 4, 4, 2, 8, 0, 0) == 1
    assert call(fake, fake, fake, 4, 4, 2, 7, 1, 0) == 1        # ldR < nb * S


def test_selftest_limit_validation(lib):
    assert lib.tdm_selftest_wait_timeout(0, None) == 1
    assert lib.tdm_selftest_wait_timeout((1 << 31) + 1, None) == 1
    assert lib.tdm_selftest_group_timeout(0, None) == 1
    assert lib.tdm_selftest_group_timeout((1 << 24) + 1, None) == 1
