"""CPU-side checks of the C-ABI library: it builds, loads, exports every entry
point declared in include/hac.h, and rejects bad arguments before touching
the device (no compute call runs here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2106_04727_gb300 import hac

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hac_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("hac_create", "hac_run", "hac_dendrogram", "hac_destroy", "hac_stats",
                 "hac_strerror", "hac_create_device", "hac_merge_rounds", "hac_default_opts"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = hac.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    assert ctypes.sizeof(hac.hac_merge) == 32
    assert ctypes.sizeof(hac.hac_opts) == 40
    assert hac.MERGE_DTYPE.itemsize == 32


def test_default_opts_and_strerror():
    o = hac.hac_default_opts()
    assert o.precision == 0 and o.cache_slots == 0 and o.max_rounds == 0 and not o.stream
    for code in range(0, -8, -1):
        assert hac.hac_strerror(code) != "unknown status"
    assert hac.hac_strerror(-99) == "unknown status"


@pytest.mark.parametrize("bad", ["nan", "inf", "d0", "d17", "n0", "null"])
def test_create_rejects_bad_arguments_on_host(bad):
    """Argument checks run before any CUDA call, so they work without a GPU."""
    lib = hac.load()
    X = np.random.default_rng(0).normal(size=(10, 3))
    n, d = X.shape
    if bad == "nan":
        X[3, 1] = np.nan
    if bad == "inf":
        X[0, 0] = np.inf
    if bad == "d0":
        d = 0
    if bad == "d17":
        X = np.zeros((10, 17))
        d = 17
    if bad == "n0":
        n = 0
    h = ctypes.c_void_p()
    ptr = None if bad == "null" else X.ctypes.data_as(ctypes.c_void_p)
    rc = lib.hac_create(ptr, n, d, hac.F64, hac.WARD, ctypes.byref(h))
    assert rc == hac.HAC_EINVAL and not h.value


def test_bad_enums_rejected():
    lib = hac.load()
    X = np.zeros((4, 2))
    h = ctypes.c_void_p()
    assert lib.hac_create(X.ctypes.data_as(ctypes.c_void_p), 4, 2, 7, hac.WARD,
                          ctypes.byref(h)) == hac.HAC_EINVAL
    for lk in (-1, 4):
        assert lib.hac_create(X.ctypes.data_as(ctypes.c_void_p), 4, 2, hac.F64, lk,
                              ctypes.byref(h)) == hac.HAC_EINVAL


def test_null_handle_calls():
    lib = hac.load()
    w = ctypes.c_int64()
    assert lib.hac_run(None, None) == hac.HAC_EINVAL
    assert lib.hac_dendrogram(None, None, 0, ctypes.byref(w)) == hac.HAC_EINVAL
    lib.hac_destroy(None)
