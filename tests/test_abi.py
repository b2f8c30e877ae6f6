"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/wl.h declares; host-side argument checks (no GPU)."""
import ctypes
import os
import re

import numpy as np

from paper_2601_11338_gb300 import wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "wl.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(wl_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("wl_build", "wl_degrees", "wl_apply", "wl_expmv", "wl_trace", "wl_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    L = wl.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    for code in range(-12, 1):
        s = wl.status_string(code)
        assert s and s != "unknown status"
    assert wl.status_string(-99) == "unknown status"


def test_build_rejects_bad_arguments_before_touching_the_gpu():
    L = wl.lib()
    h = ctypes.c_void_p()
    p = wl.make_params()
    # NULL csr
    assert L.wl_build(None, 0, ctypes.byref(p), ctypes.byref(h), None) == wl.WL_ERR_INVALID_ARG
    # negative size
    A = wl.wl_csr(-1, 0, None, None)
    assert L.wl_build(ctypes.byref(A), 0, ctypes.byref(p), ctypes.byref(h), None) == wl.WL_ERR_INVALID_ARG
    # bad variant / mu out of range
    rp = np.zeros(3, dtype=np.int32)
    A = wl.wl_csr(2, 0, rp.ctypes.data, None)
    assert L.wl_build(ctypes.byref(A), 7, ctypes.byref(p), ctypes.byref(h), None) == wl.WL_ERR_INVALID_ARG
    p2 = wl.make_params(mu=1.5)
    assert L.wl_build(ctypes.byref(A), wl.WL_BTDW, ctypes.byref(p2), ctypes.byref(h), None) == wl.WL_ERR_INVALID_ARG
    # unknown matrix function
    p3 = wl.make_params(f=9)
    assert L.wl_build(ctypes.byref(A), wl.WL_NBT, ctypes.byref(p3), ctypes.byref(h), None) == wl.WL_ERR_INVALID_ARG
    # unknown precision, reorthogonalisation mode or Gram kernel, negative or non-finite shift
    for bad in (wl.make_params(prec=5), wl.make_params(reorth=2), wl.make_params(shift=-1.0),
                wl.make_params(shift=float("nan")), wl.make_params(shift=float("inf")), wl.make_params(gram=2),
                wl.make_params(gram=-1)):
        assert L.wl_build(ctypes.byref(A), wl.WL_NBT, ctypes.byref(bad), ctypes.byref(h), None) == wl.WL_ERR_INVALID_ARG
    assert h.value is None


def test_null_handle_calls_are_rejected():
    L = wl.lib()
    assert L.wl_degrees(None, None, None) == wl.WL_ERR_INVALID_ARG
    assert L.wl_apply(None, None, 0, 0, None, 0, None) == wl.WL_ERR_INVALID_ARG
    assert L.wl_expmv(None, None, 0, 0, None, 0, None, 0, None) == wl.WL_ERR_INVALID_ARG
    L.wl_destroy(None)


def test_wait_selftest_rejects_bad_counts_before_touching_the_gpu():
    assert wl.wl_selftest_bounded_wait(-1) == wl.WL_ERR_INVALID_ARG
    assert wl.wl_selftest_bounded_wait(5000) == wl.WL_ERR_INVALID_ARG
