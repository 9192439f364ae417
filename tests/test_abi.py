"""CPU-side checks of the C-ABI library: it builds, loads, exports every entry
point declared in include/hac.h, and rejects bad arguments before touching
the device (no compute call runs here)."""
import ctypes
import os
import re
import shutil
import subprocess

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


def test_header_is_plain_c_and_matches_the_binding(tmp_path):
    """A C11 program built against include/hac.h alone (gcc -pedantic
    -Werror) and linked with the library: every declared entry point
    resolves, and every struct's size and field offsets equal the binding's
    ctypes layout."""
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    lib = hac.lib_path()
    if not os.path.exists(lib):
        hac.load()
    structs = {"hac_merge": hac.hac_merge, "hac_opts": hac.hac_opts,
               "hac_stats_t": hac.hac_stats_t, "hac_server_stats_t": hac.hac_server_stats_t}
    body = []
    for name, cls in structs.items():
        body.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            body.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    body.append("  void (*volatile fp)(void);")
    for fn in _declared():
        body.append(f"  fp = (void (*)(void)){fn};")
        body.append(f'  printf("fn {fn} %d\\n", fp != 0);')
    src = tmp_path / "abi.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"hac.h\"\n"
                   "int main(void) {\n" + "\n".join(body) + "\n  return 0;\n}\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    lib, f"-Wl,-rpath,{libdir}"], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
    for fn in _declared():
        assert got[f"fn {fn}"] == "1", fn


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
