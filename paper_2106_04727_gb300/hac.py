"""Thin Python binding of the C ABI in include/hac.h (argument marshalling only).

Every function here forwards to the same-named ``extern "C"`` entry point of
``libhac.so``; all clustering work runs in the library's CUDA kernels.  There
is no CPU fallback: importing works anywhere, but the first call raises if the
library cannot be loaded or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

COMPLETE, AVERAGE, WARD, AVERAGE_SQ = 0, 1, 2, 3
LINKAGES = {"complete": COMPLETE, "average": AVERAGE, "ward": WARD, "average_sq": AVERAGE_SQ}
F32, F64 = 0, 1
PREC_F64, PREC_F32_RECHECK = 0, 1

HAC_OK, HAC_EINVAL, HAC_ENOMEM, HAC_EDEVICE = 0, -1, -2, -3
HAC_ETIMEOUT, HAC_EPENDING, HAC_ECAP, HAC_EINTERNAL = -4, -5, -6, -7
HAC_ECANCELED = -8


class hac_merge(ctypes.Structure):
    _fields_ = [("cid_a", ctypes.c_int64), ("cid_b", ctypes.c_int64),
                ("height", ctypes.c_double), ("size", ctypes.c_int64)]


class hac_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cache_slots", ctypes.c_int),
                ("max_rounds", ctypes.c_int64), ("timeout_s", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("flags", ctypes.c_int)]


class hac_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("rounds", "merges", "nn_searches", "cluster_pairs",
                                              "point_pairs", "nodes_visited", "rechecks")] + \
               [(k, ctypes.c_double) for k in ("ms_init", "ms_nn", "ms_merge", "ms_update",
                                               "ms_total")] + [("device_bytes", ctypes.c_int64),
               ("ms_query", ctypes.c_double)] + \
               [(k, ctypes.c_int64) for k in ("query_launches", "query_bytes", "leaf_tests",
                                              "kernel_launches", "cache_hits",
                                              "cache_lw_entries")] + \
               [("ms_big", ctypes.c_double), ("big_point_pairs", ctypes.c_int64),
                ("big_launches", ctypes.c_int64), ("naive_pairs", ctypes.c_int64)] + \
               [(k, ctypes.c_int64) for k in ("dense_k", "dense_rounds", "dense_point_pairs",
                                              "dense_rechecks")] + [("ms_dense", ctypes.c_double)]


class hac_server_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("engines", "rounds", "admitted", "completed",
                                              "queued", "resident", "max_resident",
                                              "device_bytes", "kernel_launches")] + \
               [(k, ctypes.c_double) for k in ("ms_admit", "ms_rounds", "ms_harvest")]


MERGE_DTYPE = np.dtype([("cid_a", np.int64), ("cid_b", np.int64), ("height", np.float64),
                        ("size", np.int64)])

_lib = None
_lock = threading.Lock()


class HacError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {hac_strerror(code)} ({code})")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhac.so (building it in-tree if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libhac.so not found at {path}; run build()")
        L = ctypes.CDLL(path)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.hac_default_opts.argtypes = [ctypes.POINTER(hac_opts)]
        L.hac_default_opts.restype = None
        L.hac_create.argtypes = [P, i64, i32, i32, i32, ctypes.POINTER(P)]
        L.hac_create.restype = i32
        L.hac_create_device.argtypes = [P, i64, i32, i32, i32, ctypes.POINTER(P)]
        L.hac_create_device.restype = i32
        L.hac_run.argtypes = [P, ctypes.POINTER(hac_opts)]
        L.hac_run.restype = i32
        L.hac_dendrogram.argtypes = [P, P, i64, ctypes.POINTER(i64)]
        L.hac_dendrogram.restype = i32
        L.hac_merge_rounds.argtypes = [P, P, i64, ctypes.POINTER(i64)]
        L.hac_merge_rounds.restype = i32
        L.hac_stats.argtypes = [P, ctypes.POINTER(hac_stats_t)]
        L.hac_stats.restype = i32
        L.hac_destroy.argtypes = [P]
        L.hac_destroy.restype = None
        L.hac_strerror.argtypes = [i32]
        L.hac_strerror.restype = ctypes.c_char_p
        L.hac_run_static.argtypes = [P, i64, i32, i32, i32, ctypes.POINTER(hac_opts), P, i64]
        L.hac_run_static.restype = i32
        u64, f64 = ctypes.c_uint64, ctypes.c_double
        L.hac_server_create.argtypes = [i64, ctypes.POINTER(hac_opts), ctypes.POINTER(P)]
        L.hac_server_create.restype = i32
        L.hac_submit.argtypes = [P, P, i64, i32, i32, i32, f64, ctypes.POINTER(u64)]
        L.hac_submit.restype = i32
        L.hac_cancel.argtypes = [P, u64]
        L.hac_cancel.restype = i32
        L.hac_poll.argtypes = [P, u64, P, i64, ctypes.POINTER(i64), ctypes.POINTER(f64)]
        L.hac_poll.restype = i32
        L.hac_server_wait.argtypes = [P, u64, f64]
        L.hac_server_wait.restype = i32
        L.hac_server_stats.argtypes = [P, ctypes.POINTER(hac_server_stats_t)]
        L.hac_server_stats.restype = i32
        L.hac_server_destroy.argtypes = [P]
        L.hac_server_destroy.restype = None
        L.hac_run_batch.argtypes = [ctypes.POINTER(P), i32, ctypes.POINTER(hac_opts)]
        L.hac_run_batch.restype = i32
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc != HAC_OK:
        raise HacError(rc, what)


def hac_strerror(code: int) -> str:
    return load().hac_strerror(int(code)).decode()


def hac_default_opts() -> hac_opts:
    o = hac_opts()
    load().hac_default_opts(ctypes.byref(o))
    return o


def _lk(linkage) -> int:
    return LINKAGES[linkage] if isinstance(linkage, str) else int(linkage)


def hac_create(points: np.ndarray, linkage) -> ctypes.c_void_p:
    """hac_create with host points (float32 or float64, shape (n, d))."""
    X = np.ascontiguousarray(points)
    if X.dtype not in (np.float32, np.float64) or X.ndim != 2:
        raise ValueError("points must be a float32/float64 (n, d) array")
    h = ctypes.c_void_p()
    rc = load().hac_create(X.ctypes.data_as(ctypes.c_void_p), X.shape[0], X.shape[1],
                           F32 if X.dtype == np.float32 else F64, _lk(linkage), ctypes.byref(h))
    _check(rc, "hac_create")
    return h


def hac_create_device(dev_ptr: int, n: int, d: int, dtype, linkage) -> ctypes.c_void_p:
    """hac_create_device with a device pointer (e.g. torch ``t.data_ptr()``)."""
    dt = F32 if np.dtype(dtype) == np.float32 else F64
    h = ctypes.c_void_p()
    rc = load().hac_create_device(ctypes.c_void_p(dev_ptr), n, d, dt, _lk(linkage), ctypes.byref(h))
    _check(rc, "hac_create_device")
    return h


HAC_FLAG_NO_PRUNE = 1


def hac_run(h, precision: int = PREC_F64, cache_slots: int = 0, max_rounds: int = 0,
            timeout_s: float = 0.0, stream: int | None = None, no_prune: bool = False) -> int:
    """hac_run; returns the status code (raises on device/internal errors).
    ``no_prune`` sets HAC_FLAG_NO_PRUNE (the range-query ablation)."""
    o = hac_default_opts()
    o.precision, o.cache_slots, o.max_rounds, o.timeout_s = precision, cache_slots, max_rounds, timeout_s
    o.stream = stream
    o.flags = HAC_FLAG_NO_PRUNE if no_prune else 0
    rc = load().hac_run(h, ctypes.byref(o))
    if rc in (HAC_EDEVICE, HAC_EINTERNAL):
        raise HacError(rc, "hac_run")
    return rc


def hac_dendrogram(h, n: int) -> np.ndarray:
    out = np.zeros(max(n - 1, 1), dtype=MERGE_DTYPE)
    w = ctypes.c_int64()
    _check(load().hac_dendrogram(h, out.ctypes.data_as(ctypes.c_void_p), len(out),
                                 ctypes.byref(w)), "hac_dendrogram")
    return out[: w.value]


def hac_merge_rounds(h, n: int) -> np.ndarray:
    out = np.zeros(max(n - 1, 1), dtype=np.int32)
    w = ctypes.c_int64()
    _check(load().hac_merge_rounds(h, out.ctypes.data_as(ctypes.c_void_p), len(out),
                                   ctypes.byref(w)), "hac_merge_rounds")
    return out[: w.value]


def hac_stats(h) -> dict:
    s = hac_stats_t()
    _check(load().hac_stats(h, ctypes.byref(s)), "hac_stats")
    return {k: getattr(s, k) for k, _ in hac_stats_t._fields_}


def hac_destroy(h) -> None:
    if h:
        load().hac_destroy(h)


HAC_STATIC_MAX_N = 4096


def hac_run_static(dev_points: int, n: int, d: int, dtype, linkage, dev_out: int, cap: int,
                   precision: int = PREC_F64, stream: int | None = None) -> int:
    """hac_run_static: the whole clustering with no device allocation.

    For callers that cannot call cudaMalloc when they need a dendrogram (a
    memory pool that already owns the GPU, or code that must not risk the
    device-wide synchronisation of cudaMalloc/cudaFree).  ``dev_points`` and
    ``dev_out`` are device pointers owned by the caller (``dev_out`` holds at
    least n - 1 records of MERGE_DTYPE); working memory comes from a fixed
    array inside the library.  Returns the status code.  Calls share that
    array, so calls that overlap on the GPU must be serialised by the caller.
    """
    o = hac_default_opts()
    o.precision = precision
    o.stream = stream
    dt = F32 if np.dtype(dtype) == np.float32 else F64
    return load().hac_run_static(ctypes.c_void_p(dev_points), n, d, dt, _lk(linkage),
                                 ctypes.byref(o), ctypes.c_void_p(dev_out), cap)


def cluster(points: np.ndarray, linkage, precision: int = PREC_F64, with_rounds: bool = True,
            **run_kw) -> dict:
    """create -> run -> dendrogram -> destroy, returned in the oracle's dict
    layout: a, b, h, size (and round, stats)."""
    X = np.ascontiguousarray(points)
    h = hac_create(X, linkage)
    try:
        rc = hac_run(h, precision=precision, **run_kw)
        _check(rc, "hac_run")
        m = hac_dendrogram(h, len(X))
        out = dict(a=m["cid_a"].copy(), b=m["cid_b"].copy(), h=m["height"].copy(),
                   size=m["size"].copy())
        if with_rounds:
            out["round"] = hac_merge_rounds(h, len(X)).astype(np.int64)
        out["stats"] = hac_stats(h)
        return out
    finally:
        hac_destroy(h)


# ---------------------------------------------------------------------------
# serving (continuous batching of independent requests)
# ---------------------------------------------------------------------------

def hac_server_create(points_per_engine: int, precision: int = PREC_F64,
                      cache_slots: int = 0) -> ctypes.c_void_p:
    o = hac_default_opts()
    o.precision = precision
    o.cache_slots = cache_slots
    srv = ctypes.c_void_p()
    _check(load().hac_server_create(points_per_engine, ctypes.byref(o), ctypes.byref(srv)),
           "hac_server_create")
    return srv


def hac_submit(srv, points: np.ndarray, linkage, timeout_s: float = 0.0) -> int:
    """Queue one request (host points, float32/float64 (n, d)); returns its ticket."""
    X = np.ascontiguousarray(points)
    if X.dtype not in (np.float32, np.float64) or X.ndim != 2:
        raise ValueError("points must be a float32/float64 (n, d) array")
    t = ctypes.c_uint64()
    _check(load().hac_submit(srv, X.ctypes.data_as(ctypes.c_void_p), X.shape[0], X.shape[1],
                             F32 if X.dtype == np.float32 else F64, _lk(linkage),
                             float(timeout_s), ctypes.byref(t)), "hac_submit")
    return t.value


def hac_cancel(srv, ticket: int) -> int:
    return load().hac_cancel(srv, ticket)


def hac_poll(srv, ticket: int, n: int):
    """(status, merges or None, latency_ms): status HAC_EPENDING while it runs."""
    out = np.zeros(max(n - 1, 1), dtype=MERGE_DTYPE)
    got = ctypes.c_int64()
    lat = ctypes.c_double()
    rc = load().hac_poll(srv, ticket, ctypes.c_void_p(out.ctypes.data), max(n - 1, 0),
                         ctypes.byref(got), ctypes.byref(lat))
    if rc != HAC_OK:
        return rc, None, (lat.value if rc != HAC_EPENDING else None)
    return rc, out[:got.value], lat.value


def hac_server_wait(srv, ticket: int, timeout_s: float = 0.0) -> int:
    return load().hac_server_wait(srv, ticket, float(timeout_s))


def hac_server_stats(srv) -> dict:
    st = hac_server_stats_t()
    rc = load().hac_server_stats(srv, ctypes.byref(st))
    d = {k: getattr(st, k) for k, _ in hac_server_stats_t._fields_}
    d["status"] = rc
    return d


def hac_server_destroy(srv) -> None:
    if srv:
        load().hac_server_destroy(srv)


def result_dict(m: np.ndarray) -> dict:
    """A merge array in the oracle's dict layout."""
    return dict(a=m["cid_a"].copy(), b=m["cid_b"].copy(), h=m["height"].copy(),
                size=m["size"].copy())


def hac_run_batch(handles, precision: int = PREC_F64, cache_slots: int = 0,
                  timeout_s: float = 0.0) -> int:
    """hac_run for several handles at once (one engine per kind); returns the status."""
    o = hac_default_opts()
    o.precision = precision
    o.cache_slots = cache_slots
    o.timeout_s = timeout_s
    arr = (ctypes.c_void_p * max(len(handles), 1))(*[h.value for h in handles])
    return load().hac_run_batch(arr, len(handles), ctypes.byref(o))
