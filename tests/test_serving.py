"""Serving: many independent requests batched on one GPU (continuous batching).

Each request's dendrogram from the server must be the one a lone run of the
same request gives (same merges, heights within the stated tolerance), and,
for small requests, the oracle's.  Requests that arrive while others are on
the GPU join at the next round; requests that do not fit wait until ids free
up; cancelled and timed-out requests leave without disturbing the others.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2106_04727_gb300 import hac, inputs

pytestmark = pytest.mark.gpu

RTOL64 = 1e-9
RTOL32 = 1e-5


def _rtol(lk, prec):
    return RTOL64 if prec == hac.PREC_F64 or lk == hac.WARD else RTOL32


def _collect(srv, tickets, ns, timeout=300.0):
    out = {}
    for t, n in zip(tickets, ns):
        assert hac.hac_server_wait(srv, t, timeout) == hac.HAC_OK
        rc, m, lat = hac.hac_poll(srv, t, n)
        assert rc == hac.HAC_OK, hac.hac_strerror(rc)
        assert lat is not None and lat >= 0
        out[t] = m
    return out


def _alone(X, lk, prec, slots):
    return hac.cluster(X, lk, precision=prec, with_rounds=False, cache_slots=slots)


@pytest.mark.parametrize("prec,slots", [(hac.PREC_F64, 0), (hac.PREC_F32_RECHECK, 64)],
                         ids=["f64", "f32recheck_cache"])
def test_each_result_same_alone_and_in_the_mix(prec, slots):
    reqs = inputs.serving_requests(40, seed=11, n_lo=64, n_hi=2500)
    pts = [inputs.request_points(r) for r in reqs]
    srv = hac.hac_server_create(1 << 15, precision=prec, cache_slots=slots)
    try:
        tickets = [hac.hac_submit(srv, X, r["linkage"]) for r, X in zip(reqs, pts)]
        got = _collect(srv, tickets, [r["n"] for r in reqs])
        st = hac.hac_server_stats(srv)
    finally:
        hac.hac_server_destroy(srv)
    assert st["status"] == hac.HAC_OK
    assert st["admitted"] == st["completed"] == len(reqs)
    assert st["max_resident"] >= 2  # requests of one kind shared rounds
    for r, X, t in zip(reqs, pts, tickets):
        lk = r["linkage"]
        mixed = hac.result_dict(got[t])
        alone = _alone(X, lk, prec, slots)
        c = oracle.compare(mixed, alone, rtol=_rtol(lk, prec))
        assert c["ok"], (r, c)
        if r["n"] <= 1200:  # and the oracle's tree
            want = oracle.nnchain(X.astype(np.float64), lk)
            c = oracle.compare(mixed, want, rtol=_rtol(lk, prec))
            assert c["ok"], (r, c)


def test_f64_inputs_and_degenerate_requests():
    srv = hac.hac_server_create(4096)
    try:
        X1 = inputs.uniform_cube(1, 3, seed=5)
        X2 = inputs.uniform_cube(2, 3, seed=6)
        Xd = np.repeat(inputs.uniform_cube(40, 2, seed=7), 3, axis=0)  # duplicates: height 0
        X = inputs.uniform_cube(700, 5, seed=8)
        ts = [hac.hac_submit(srv, A, lk) for A, lk in
              ((X1, hac.WARD), (X2, hac.COMPLETE), (Xd, hac.AVERAGE), (X, hac.AVERAGE),
               (X, hac.WARD), (X, hac.COMPLETE))]
        got = _collect(srv, ts, [1, 2, len(Xd), 700, 700, 700])
        with pytest.raises(hac.HacError) as e:
            hac.hac_submit(srv, inputs.uniform_cube(5000, 2, seed=9), hac.WARD)
        assert e.value.code == hac.HAC_ENOMEM
        bad = X.copy()
        bad[3, 1] = np.nan
        with pytest.raises(hac.HacError) as e:
            hac.hac_submit(srv, bad, hac.WARD)
        assert e.value.code == hac.HAC_EINVAL
        rc, _, _ = hac.hac_poll(srv, ts[0], 1)
        assert rc == hac.HAC_EINVAL  # released by the first poll
    finally:
        hac.hac_server_destroy(srv)
    assert len(got[ts[0]]) == 0
    assert len(got[ts[1]]) == 1 and got[ts[1]]["cid_a"][0] == 0 and got[ts[1]]["cid_b"][0] == 1
    for t, A, lk in ((ts[2], Xd, "average"), (ts[3], X, "average"), (ts[4], X, "ward"),
                     (ts[5], X, "complete")):
        c = oracle.compare(hac.result_dict(got[t]), oracle.nnchain(A, lk), rtol=RTOL64)
        assert c["ok"], (lk, c)


def test_admission_waits_for_free_ids():
    # total n well above the engine's capacity: requests queue until ids free
    cap = 4096
    rng = np.random.default_rng(3)
    ns = [int(v) for v in rng.integers(900, 3500, size=14)]
    pts = [inputs.gaussian_mixture(n, 2, 6, seed=100 + i) for i, n in enumerate(ns)]
    srv = hac.hac_server_create(cap)
    try:
        ts = [hac.hac_submit(srv, X, hac.WARD) for X in pts]
        st0 = hac.hac_server_stats(srv)
        got = _collect(srv, ts, ns)
        st = hac.hac_server_stats(srv)
    finally:
        hac.hac_server_destroy(srv)
    assert sum(ns) > 2 * cap
    assert st0["queued"] + st0["resident"] + st0["completed"] == len(ns)
    assert st["admitted"] == st["completed"] == len(ns) and st["queued"] == 0
    assert st["max_resident"] >= 2
    for X, t in zip(pts, ts):
        c = oracle.compare(hac.result_dict(got[t]), _alone(X, hac.WARD, hac.PREC_F64, 0),
                           rtol=RTOL64)
        assert c["ok"], c


def _wait_rounds(srv, k, limit=60.0):
    t0 = time.time()
    while hac.hac_server_stats(srv)["rounds"] < k:
        assert time.time() - t0 < limit
        time.sleep(0.001)


def test_late_arrivals_join_running_work():
    # a long request is on the GPU; small ones of the same kind submitted
    # afterwards are admitted at the next round and finish first
    big = inputs.gaussian_mixture(40000, 2, 16, seed=21).astype(np.float64)
    small = [inputs.gaussian_mixture(n, 2, 4, seed=30 + n).astype(np.float64)
             for n in (300, 800, 150, 1200)]
    srv = hac.hac_server_create(1 << 16, cache_slots=64)
    try:
        tb = hac.hac_submit(srv, big, hac.AVERAGE)
        _wait_rounds(srv, 2)
        ts = [hac.hac_submit(srv, X, hac.AVERAGE) for X in small]
        got = _collect(srv, ts, [len(X) for X in small])
        rc_big_meanwhile, _, _ = hac.hac_poll(srv, tb, len(big))
        st = hac.hac_server_stats(srv)
        gb = _collect(srv, [tb], [len(big)])[tb]
    finally:
        hac.hac_server_destroy(srv)
    assert rc_big_meanwhile == hac.HAC_EPENDING
    assert st["engines"] == 1 and st["max_resident"] >= 2
    for X, t in zip(small, ts):
        c = oracle.compare(hac.result_dict(got[t]), oracle.nnchain(X, "average"), rtol=RTOL64)
        assert c["ok"], c
    c = oracle.compare(hac.result_dict(gb), _alone(big, hac.AVERAGE, hac.PREC_F64, 64),
                       rtol=RTOL64)
    assert c["ok"], c


def test_cancel_and_deadline_leave_the_engine_usable():
    big = inputs.gaussian_mixture(40000, 2, 16, seed=41).astype(np.float64)
    X = inputs.gaussian_mixture(900, 2, 5, seed=42).astype(np.float64)
    srv = hac.hac_server_create(1 << 16, cache_slots=64)
    try:
        # resident request cancelled mid-flight
        t1 = hac.hac_submit(srv, big, hac.AVERAGE)
        _wait_rounds(srv, 2)
        assert hac.hac_cancel(srv, t1) == hac.HAC_OK
        assert hac.hac_server_wait(srv, t1, 120.0) == hac.HAC_OK
        assert hac.hac_poll(srv, t1, len(big))[0] == hac.HAC_ECANCELED
        # resident request past its deadline
        t2 = hac.hac_submit(srv, big, hac.AVERAGE, timeout_s=0.05)
        assert hac.hac_server_wait(srv, t2, 120.0) == hac.HAC_OK
        assert hac.hac_poll(srv, t2, len(big))[0] == hac.HAC_ETIMEOUT
        # a queued request (no room behind a resident one) cancelled at once
        t3 = hac.hac_submit(srv, big, hac.AVERAGE)
        t4 = hac.hac_submit(srv, big, hac.AVERAGE)
        assert hac.hac_cancel(srv, t4) == hac.HAC_OK
        assert hac.hac_poll(srv, t4, len(big))[0] == hac.HAC_ECANCELED
        assert hac.hac_cancel(srv, t3) == hac.HAC_OK
        # the engine still clusters correctly afterwards
        t5 = hac.hac_submit(srv, X, hac.AVERAGE)
        got = _collect(srv, [t5], [len(X)])[t5]
        assert hac.hac_server_wait(srv, t3, 120.0) == hac.HAC_OK
        assert hac.hac_poll(srv, t3, len(big))[0] in (hac.HAC_ECANCELED, hac.HAC_OK)
        st = hac.hac_server_stats(srv)
    finally:
        hac.hac_server_destroy(srv)
    assert st["status"] == hac.HAC_OK and st["resident"] == 0
    c = oracle.compare(hac.result_dict(got), oracle.nnchain(X, "average"), rtol=RTOL64)
    assert c["ok"], c


def test_destroy_with_requests_in_flight():
    srv = hac.hac_server_create(1 << 16, cache_slots=64)
    for s in range(3):
        hac.hac_submit(srv, inputs.gaussian_mixture(30000, 3, 8, seed=50 + s), hac.COMPLETE)
    _wait_rounds(srv, 1)
    hac.hac_server_destroy(srv)  # stops after the current round, frees everything
    # the device is still usable
    X = inputs.uniform_cube(300, 2, seed=1)
    c = oracle.compare(hac.cluster(X, "ward", with_rounds=False), oracle.nnchain(X, "ward"),
                       rtol=RTOL64)
    assert c["ok"], c


def _round_sets(a, b, rounds):
    out = {}
    for x, y, r in zip(a, b, rounds):
        out.setdefault(int(r), set()).add((int(x), int(y)))
    return out


@pytest.mark.parametrize("prec,slots", [(hac.PREC_F64, 0), (hac.PREC_F32_RECHECK, 64)],
                         ids=["f64", "f32recheck_cache"])
def test_run_batch_matches_hac_run(prec, slots):
    reqs = inputs.serving_requests(18, seed=23, n_lo=2, n_hi=3000)
    pts = [inputs.request_points(r) for r in reqs]
    pts += [inputs.uniform_cube(1, 2, seed=1), inputs.uniform_cube(500, 3, seed=2)]
    lks = [r["linkage"] for r in reqs] + [hac.WARD, hac.COMPLETE]
    hs = [hac.hac_create(X, lk) for X, lk in zip(pts, lks)]
    try:
        assert hac.hac_run_batch(hs, precision=prec, cache_slots=slots) == hac.HAC_OK
        for h, X, lk in zip(hs, pts, lks):
            n = len(X)
            m = hac.hac_dendrogram(h, n)
            rd = hac.hac_merge_rounds(h, n)
            alone = hac.cluster(X, lk, precision=prec, cache_slots=slots)
            got = hac.result_dict(m)
            c = oracle.compare(got, alone, rtol=_rtol(lk, prec))
            assert c["ok"], (n, lk, c)
            assert _round_sets(m["cid_a"], m["cid_b"], rd) == \
                _round_sets(alone["a"], alone["b"], alone["round"])
            assert hac.hac_stats(h)["rounds"] == alone["stats"]["rounds"]
        # the handles stay usable for a plain run
        assert hac.hac_run(hs[-1], precision=prec, cache_slots=slots) == hac.HAC_OK
        assert hac.hac_run_batch([hs[0], hs[0]]) == hac.HAC_EINVAL
    finally:
        for h in hs:
            hac.hac_destroy(h)


def test_poll_capacity_cancel_after_done_and_bad_arguments():
    X = inputs.gaussian_mixture(500, 3, 4, seed=61).astype(np.float64)
    srv = hac.hac_server_create(4096)
    try:
        t = hac.hac_submit(srv, X, hac.AVERAGE_SQ)
        assert hac.hac_server_wait(srv, t, 120.0) == hac.HAC_OK
        # too small an output buffer keeps the ticket
        out = np.zeros(10, dtype=hac.MERGE_DTYPE)
        import ctypes
        got = ctypes.c_int64()
        rc = hac.load().hac_poll(srv, t, ctypes.c_void_p(out.ctypes.data), 10, ctypes.byref(got),
                                 None)
        assert rc == hac.HAC_ECAP
        # cancelling a finished request keeps its result
        assert hac.hac_cancel(srv, t) == hac.HAC_OK
        rc, m, lat = hac.hac_poll(srv, t, len(X))
        assert rc == hac.HAC_OK and len(m) == len(X) - 1
        c = oracle.compare(hac.result_dict(m), oracle.nnchain(X, "average_sq"), rtol=RTOL64)
        assert c["ok"], c
        # unknown tickets and bad arguments
        assert hac.hac_cancel(srv, 987654) == hac.HAC_EINVAL
        assert hac.hac_server_wait(srv, 987654, 0.1) == hac.HAC_EINVAL
        with pytest.raises(hac.HacError) as e:
            hac.hac_submit(srv, np.zeros((4, 17)), hac.WARD)  # d > 16
        assert e.value.code == hac.HAC_EINVAL
        with pytest.raises(hac.HacError) as e:
            hac.hac_submit(srv, X, 9)  # unknown linkage
        assert e.value.code == hac.HAC_EINVAL
        st = hac.hac_server_stats(srv)
        assert st["status"] == hac.HAC_OK and st["queued"] == 0 and st["resident"] == 0
    finally:
        hac.hac_server_destroy(srv)


def test_server_rejects_bad_options():
    import ctypes
    o = hac.hac_default_opts()
    o.precision = 7
    srv = ctypes.c_void_p()
    assert hac.load().hac_server_create(1024, ctypes.byref(o), ctypes.byref(srv)) == hac.HAC_EINVAL
    assert hac.load().hac_server_create(1, None, ctypes.byref(srv)) == hac.HAC_EINVAL


def test_fp32_server_refuses_huge_coordinates():
    """An FP32 + re-score server takes FP32 copies below 2^40 (FP32 input:
    the coordinates; FP64 input: the recentred ones); an FP64 server takes
    anything finite."""
    X = np.random.default_rng(5).normal(size=(50, 3)) * 1e13
    srv = hac.hac_server_create(1 << 12, precision=hac.PREC_F32_RECHECK)
    try:
        for Y in (X, X.astype(np.float32)):
            with pytest.raises(hac.HacError) as ex:
                hac.hac_submit(srv, Y, "ward")
            assert ex.value.code == hac.HAC_EINVAL
        # a large offset with a small extent is fine for FP64 input
        t = hac.hac_submit(srv, X * 1e-13 + 1e15, "ward")
        assert hac.hac_server_wait(srv, t, 60.0) == hac.HAC_OK
    finally:
        hac.hac_server_destroy(srv)
    srv = hac.hac_server_create(1 << 12, precision=hac.PREC_F64)
    try:
        t = hac.hac_submit(srv, X, "ward")
        assert hac.hac_server_wait(srv, t, 60.0) == hac.HAC_OK
        rc, m, _ = hac.hac_poll(srv, t, len(X))
        assert rc == hac.HAC_OK and len(m) == len(X) - 1
    finally:
        hac.hac_server_destroy(srv)
