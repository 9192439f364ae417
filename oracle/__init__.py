"""CPU oracle for NN-chain HAC -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never loads it; the two
share no code.  The arithmetic lives in ``hac_oracle.c`` (plain FP64 C, see its
header for the passages of the paper each function follows); this module
compiles it with gcc and wraps it with ctypes, and holds the dendrogram
comparison helpers the tests use.

A dendrogram here is a dict of numpy arrays ``a, b, h, size`` (and ``round``
where known): merge ``t`` joined the clusters with ids ``a[t] < b[t]`` at
height ``h[t]`` into a cluster of ``size[t]`` points.  Cluster id = smallest
input index in the cluster (Section 1, footnote on the example).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

COMPLETE, AVERAGE, WARD, AVERAGE_SQ = 0, 1, 2, 3
LINKAGES = {"complete": COMPLETE, "average": AVERAGE, "ward": WARD, "average_sq": AVERAGE_SQ}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hac_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_PC_SRC = os.path.join(_HERE, "hac_parchain_cpu.c")
_PC_SO = os.path.join(_BUILD, "libparchain_cpu.so")
_lock = threading.Lock()
_lib = None
_pclib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: plain IEEE FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def build_parchain_cpu(force: bool = False) -> str:
    """Compile the multithreaded CPU NN-chain (gcc, pthreads, plain FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_PC_SO) or os.path.getmtime(_PC_SO) < os.path.getmtime(_PC_SRC):
        tmp = _PC_SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-pthread", "-o", tmp, _PC_SRC, "-lm"])
        os.replace(tmp, _PC_SO)
    return _PC_SO


def parchain_cpu(X, linkage, threads: int = 0, timeout_s: float = 0.0) -> dict:
    """Algorithm 1 on the host cores (hac_parchain_cpu.c): FP64, linear memory,
    kd-tree range queries.  threads = 0: every core.  Returns the oracle's
    dict layout (a, b, h, size, round) in merge order, plus n_rounds,
    point_pairs, seconds, threads and complete (False when timeout_s stopped
    it between rounds; then only the merges made are returned)."""
    global _pclib
    X = _pts(X)
    n, d = X.shape
    with _lock:
        if _pclib is None:
            lib = ctypes.CDLL(build_parchain_cpu())
            P = ctypes.c_void_p
            lib.parchain_cpu.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, P, P, P, P, P, P]
            lib.parchain_cpu.restype = ctypes.c_int64
            _pclib = lib
    if threads <= 0:
        threads = os.cpu_count() or 1
    m = max(n - 1, 0)
    a, b, h, s = _outs(m)
    r = np.zeros(m, np.int64)
    st = np.zeros(3, np.float64)
    got = _pclib.parchain_cpu(_p(X), n, d, _lk(linkage), threads, float(timeout_s), _p(a), _p(b),
                              _p(h), _p(s), _p(r), _p(st))
    if got < 0:
        raise ValueError(f"parchain_cpu failed ({got})")
    return dict(a=a[:got], b=b[:got], h=h[:got], size=s[:got], round=r[:got],
                n_rounds=int(st[0]), point_pairs=int(st[1]), seconds=float(st[2]),
                threads=threads, complete=bool(got == m))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_nnchain.argtypes = [P, i64, i32, i32, i64, P, P, P, P]
            lib.oracle_nnchain.restype = i32
            lib.oracle_rounds.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, P, P, i64, P]
            lib.oracle_rounds.restype = i32
            lib.oracle_greedy.argtypes = [P, i64, i32, i32, P, P, P, P]
            lib.oracle_greedy.restype = i32
            lib.oracle_validate.argtypes = [P, i64, i32, i32, P, P, P, P, i64, f64, f64, f64, P]
            lib.oracle_validate.restype = i64
            lib.oracle_lw.argtypes = [i32, f64, f64, f64, f64, f64, f64]
            lib.oracle_lw.restype = f64
            lib.oracle_cluster_dist.argtypes = [i32, P, i64, P, i64, i32]
            lib.oracle_cluster_dist.restype = f64
            lib.oracle_dist_to_all.argtypes = [i32, P, i64, i32, P, i64, i64, P]
            lib.oracle_dist_to_all.restype = i32
            _lib = lib
    return _lib


def _pts(X) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim != 2:
        raise ValueError("points must be an (n, d) array")
    return X


def _lk(linkage) -> int:
    return LINKAGES[linkage] if isinstance(linkage, str) else int(linkage)


def _outs(m):
    return (np.zeros(m, np.int64), np.zeros(m, np.int64), np.zeros(m, np.float64),
            np.zeros(m, np.int64))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def nnchain(X, linkage, start: int = 0) -> dict:
    """Sequential NN-chain over the FP64 Lance-Williams matrix."""
    X = _pts(X)
    n, d = X.shape
    a, b, h, s = _outs(max(n - 1, 0))
    rc = _load().oracle_nnchain(_p(X), n, d, _lk(linkage), start, _p(a), _p(b), _p(h), _p(s))
    if rc:
        raise ValueError(f"oracle_nnchain failed ({rc})")
    return dict(a=a, b=b, h=h, size=s)


def rounds(X, linkage, log_terminals: bool = False) -> dict:
    """Algorithm 1 round by round; adds ``round`` per merge and ``n_rounds``.

    With ``log_terminals`` the (round, cid) of every nearest-neighbour search
    is returned as ``terminals`` (an (m, 2) array).
    """
    X = _pts(X)
    n, d = X.shape
    m = max(n - 1, 0)
    a, b, h, s = _outs(m)
    r = np.zeros(m, np.int64)
    nr = np.zeros(1, np.int64)
    nt = np.zeros(1, np.int64)
    cap = 4 * n + 64 if log_terminals else 0
    tr = np.zeros(max(cap, 1), np.int64)
    tc = np.zeros(max(cap, 1), np.int64)
    lib = _load()
    while True:
        rc = lib.oracle_rounds(_p(X), n, d, _lk(linkage), _p(a), _p(b), _p(h), _p(s), _p(r),
                               _p(nr), _p(tr) if cap else None, _p(tc) if cap else None,
                               cap, _p(nt))
        if rc:
            raise ValueError(f"oracle_rounds failed ({rc})")
        if not log_terminals or nt[0] <= cap:
            break
        cap = int(nt[0])
        tr = np.zeros(cap, np.int64)
        tc = np.zeros(cap, np.int64)
    out = dict(a=a, b=b, h=h, size=s, round=r, n_rounds=int(nr[0]))
    if log_terminals:
        out["terminals"] = np.stack([tr[: nt[0]], tc[: nt[0]]], axis=1)
    return out


def greedy(X, linkage) -> dict:
    """Generic algorithm, distances recomputed from the points every step."""
    X = _pts(X)
    n, d = X.shape
    a, b, h, s = _outs(max(n - 1, 0))
    rc = _load().oracle_greedy(_p(X), n, d, _lk(linkage), _p(a), _p(b), _p(h), _p(s))
    if rc:
        raise ValueError(f"oracle_greedy failed ({rc})")
    return dict(a=a, b=b, h=h, size=s)


def validate(X, linkage, dend: dict, rtol: float = 1e-9, atol_scale: float = 1e-300,
             htol: float | None = None):
    """Greedy-validity replay of ``dend``: every merge must join a pair within
    ``rtol`` (relative) of the smallest active distance, and its height must be
    within ``htol`` (default: ``rtol``) of that pair's distance.  Returns
    (first_bad, stats) where first_bad is 0 when valid and stats = (tie-zone
    merges, max relative excess over the minimum, max relative height error)."""
    htol = rtol if htol is None else htol
    X = _pts(X)
    n, d = X.shape
    a = np.ascontiguousarray(dend["a"], dtype=np.int64)
    b = np.ascontiguousarray(dend["b"], dtype=np.int64)
    h = np.ascontiguousarray(dend["h"], dtype=np.float64)
    s = np.ascontiguousarray(dend["size"], dtype=np.int64)
    st = np.zeros(3, np.float64)
    rc = _load().oracle_validate(_p(X), n, d, _lk(linkage), _p(a), _p(b), _p(h), _p(s),
                                 len(a), rtol, htol, atol_scale, _p(st))
    if rc < 0:
        raise ValueError(f"oracle_validate failed ({rc})")
    return int(rc), (int(st[0]), float(st[1]), float(st[2]))


def lw(linkage, dac, dbc, dab, na, nb, nc) -> float:
    """One Lance-Williams update (Table 2); squared distances for Ward."""
    return _load().oracle_lw(_lk(linkage), dac, dbc, dab, na, nb, nc)


def cluster_dist(linkage, A, B) -> float:
    """Linkage distance between two point sets from the points (Table 1)."""
    A, B = _pts(A), _pts(B)
    return _load().oracle_cluster_dist(_lk(linkage), _p(A), len(A), _p(B), len(B), A.shape[1])


def dist_to_all(linkage, X, label, q) -> np.ndarray:
    """Linkage distance (Table 1) from the cluster labelled q to every label of
    a labelling of X's points (NaN for q itself and for unused labels)."""
    X = _pts(X)
    label = np.ascontiguousarray(label, dtype=np.int64)
    if label.shape != (len(X),):
        raise ValueError("one label per point")
    ncl = int(label.max()) + 1 if len(label) else 1
    out = np.empty(max(ncl, int(q) + 1), np.float64)
    rc = _load().oracle_dist_to_all(_lk(linkage), _p(X), len(X), X.shape[1], _p(label),
                                    len(out), int(q), _p(out))
    if rc:
        raise ValueError(f"oracle_dist_to_all failed ({rc})")
    return out


# ----------------------------------------------------------------------------
# dendrogram helpers (structure only; no linkage arithmetic)
# ----------------------------------------------------------------------------

def canonical(dend: dict) -> dict:
    """Sort merges by (height, size, cid_a, cid_b)."""
    order = np.lexsort((dend["b"], dend["a"], dend["size"], dend["h"]))
    return {k: (v[order] if isinstance(v, np.ndarray) and v.ndim == 1 and len(v) == len(order)
                else v) for k, v in dend.items()}


def as_map(dend: dict) -> dict:
    """{(cid_a, cid_b): (height, size)}; (cid_a, cid_b) identifies a merge
    uniquely because a cid that loses a merge never appears again."""
    return {(int(a), int(b)): (float(h), int(s))
            for a, b, h, s in zip(dend["a"], dend["b"], dend["h"], dend["size"])}


def compare(got: dict, want: dict, rtol: float) -> dict:
    """Exact tree equality plus relative height error.

    Returns dict(same_tree, missing, extra, size_mismatch, max_rel_err)."""
    g, w = as_map(got), as_map(want)
    missing = [k for k in w if k not in g]
    extra = [k for k in g if k not in w]
    size_bad = [k for k in w if k in g and g[k][1] != w[k][1]]
    err = 0.0
    for k in w:
        if k in g:
            hw, hg = w[k][0], g[k][0]
            e = abs(hg - hw) / max(abs(hw), 1e-300) if hw != 0 else abs(hg)
            err = max(err, e)
    return dict(same_tree=not missing and not extra and not size_bad,
                missing=missing[:10], extra=extra[:10], size_mismatch=size_bad[:10],
                n_missing=len(missing), max_rel_err=err, ok=(not missing and not extra
                                                            and not size_bad and err <= rtol))


def check_tree(dend: dict, n: int, rtol: float = 1e-12) -> list:
    """Structural invariants: n-1 merges; a < b; every merge joins two live
    clusters whose sizes add up; one cluster of size n remains.  Heights are
    monotone along ancestry (reducibility, Section 2).  Returns a list of
    problems (empty when valid)."""
    probs = []
    m = len(dend["a"])
    if m != n - 1:
        probs.append(f"{m} merges for n={n}")
        return probs
    size = np.ones(n, np.int64)
    alive = np.ones(n, bool)
    last_h = np.full(n, -np.inf)
    order = np.argsort(np.asarray(dend["size"]), kind="stable")  # children before parents
    for t in order:
        a, b, h, s = int(dend["a"][t]), int(dend["b"][t]), float(dend["h"][t]), int(dend["size"][t])
        if not (0 <= a < b < n):
            probs.append(f"merge {t}: bad ids {a},{b}")
            continue
        if not (alive[a] and alive[b]):
            probs.append(f"merge {t}: dead cluster {a},{b}")
            continue
        if size[a] + size[b] != s:
            probs.append(f"merge {t}: sizes {size[a]}+{size[b]} != {s}")
            continue
        if h < max(last_h[a], last_h[b]) * (1 - rtol) - 1e-300:
            probs.append(f"merge {t}: height {h} below child height {max(last_h[a], last_h[b])}")
        size[a] = s
        alive[b] = False
        last_h[a] = h
    if not probs and alive.sum() != 1:
        probs.append(f"{alive.sum()} clusters remain")
    return probs
