"""The C-ABI library loads and exports every entry point include/lfd.h
declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "lfd.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^LFD_API [^;(]*?\b(lfd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_04509_gb300 import build_lib, lfd
    build_lib.build()
    return lfd.load()


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("lfd_plan_create", "lfd_render", "lfd_render_projected", "lfd_project",
              "lfd_render_host", "lfd_plan_copy_tables", "lfd_plan_copy_lists"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    from paper_2605_04509_gb300 import lfd
    assert lib.lfd_version() >= 100
    assert lib.lfd_status_string(lfd.LFD_ERR_INVALID) == b"invalid argument"
    assert lib.lfd_status_string(12345) == b"unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_2605_04509_gb300 import lfd
    h = ctypes.c_void_p()
    assert lib.lfd_plan_create(None, None, ctypes.byref(h)) == lfd.LFD_ERR_INVALID
    assert not h.value
    assert lib.lfd_plan_get_info(None, None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_render(None, None, None, 0, None, None, None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_render_host(None, None, None, 0, None, None, None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_render_host_async(None, None, None, 0, None, None, None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_render_host_wait(None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_render_backward(None, None, None, 0, None, None, None, None, None, None,
                                   None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_measure_alu_peaks(None, None, None) == lfd.LFD_ERR_INVALID
    assert lib.lfd_set_flags(None, 0) == lfd.LFD_ERR_INVALID
    p = lfd.CPanel(100, 100, 300, 0.1, 4.0, 0.0)
    o = lfd.COpts(16, 16, 8, 1, 0, (ctypes.c_float * 3)())
    assert lib.lfd_plan_create(ctypes.byref(p), ctypes.byref(o), ctypes.byref(h)) == lfd.LFD_ERR_INVALID


def test_tile_shape_limits_without_gpu(lib):
    # tiles of up to 1024 pixels, each side in [4, 64]: shapes outside are
    # rejected before any CUDA call; shapes inside pass the checks (on a
    # machine without a GPU the plan then fails at its first allocation)
    from paper_2605_04509_gb300 import lfd
    p = lfd.CPanel(256, 144, 8, 0.1, 4.0, 0.0)
    for tw, th in [(64, 17), (64, 32), (3, 16), (16, 65), (48, 24)]:
        h = ctypes.c_void_p()
        o = lfd.COpts(tw, th, 8, 1, 0, (ctypes.c_float * 3)())
        assert lib.lfd_plan_create(ctypes.byref(p), ctypes.byref(o), ctypes.byref(h)) == \
            lfd.LFD_ERR_INVALID, (tw, th)
        assert b"tile shape" in lib.lfd_last_error()
    for tw, th in [(32, 24), (32, 32), (64, 16), (4, 4)]:
        h = ctypes.c_void_p()
        o = lfd.COpts(tw, th, 8, 1, 0, (ctypes.c_float * 3)())
        rc = lib.lfd_plan_create(ctypes.byref(p), ctypes.byref(o), ctypes.byref(h))
        if rc == lfd.LFD_OK:
            lib.lfd_plan_destroy(h)
        else:
            assert b"tile shape" not in lib.lfd_last_error(), (tw, th)
