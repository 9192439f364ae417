"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Element by element on seeded inputs: every merge (cid_a, cid_b, size) must be
identical to the oracle's and heights must agree within 1e-9 relative in FP64
mode; the round in which each merge happens must match Algorithm 1 run on the
CPU.  Inputs span several 32-cluster tree leaves and levels with ragged tails,
plus the degenerate cases (n = 1, 2, duplicates, exact ties).
"""
import json
import math
import os

import numpy as np
import pytest

import dendro
import oracle
from paper_2106_04727_gb300 import hac, inputs

pytestmark = pytest.mark.gpu

LKS = ["complete", "average", "ward", "average_sq"]
PRECS = [hac.PREC_F64, hac.PREC_F32_RECHECK]
PREC_IDS = ["f64", "f32recheck"]
RTOL64 = 1e-9
RTOL32 = 1e-5   # FP32 mode: complete/average heights carry the stated FP32 bound
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture
def tree_path(monkeypatch):
    """Average linkage on the range-query search with the Section 5 cache and
    the GPU-wide big-pair kernels: the dense matrix is off (HAC_DENSE_K=0)."""
    monkeypatch.setenv("HAC_DENSE_K", "0")


def _round_sets(d):
    out = {}
    for a, b, r in zip(d["a"], d["b"], d["round"]):
        out.setdefault(int(r), set()).add((int(a), int(b)))
    return out


def _rtol(lk, prec):
    """FP64 heights everywhere except complete/average in FP32 mode, whose
    unambiguous winners keep their FP32 upper bound (<= 8e-6 relative)."""
    return RTOL64 if prec == hac.PREC_F64 or lk in ("ward", "average_sq") else RTOL32


def _assert_same(got, want, rtol=RTOL64, rounds=True):
    c = oracle.compare(got, want, rtol=rtol)
    assert c["ok"], c
    if rounds and "round" in want:
        assert _round_sets(got) == _round_sets(want)


def test_fig1_worked_example():
    with open(os.path.join(GOLDEN, "fig1_six_points.json")) as f:
        g = json.load(f)
    X = np.array(g["points"], dtype=np.float64)
    got = hac.cluster(X, g["linkage"])
    want = {i: {tuple(p) for p in ms} for i, ms in enumerate(g["round_merges"])}
    assert _round_sets(got) == want
    assert got["stats"]["rounds"] == g["n_rounds"]
    m = oracle.as_map(got)
    for k, h2 in g["squared_heights"].items():
        assert m[tuple(map(int, k.split(",")))][0] == math.sqrt(h2)
    # nearest-neighbour searches: 6 + 3 + 3 + 2 (f skips round 2)
    assert got["stats"]["nn_searches"] == sum(len(t) for t in g["round_terminals"])


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", LKS)
def test_uniform_1024_fp64(lk, prec):
    X = inputs.workload("uniform2d_1k_f64")
    _assert_same(hac.cluster(X, lk, precision=prec), oracle.rounds(X, lk), rtol=_rtol(lk, prec))


SHAPES = [(2, 2, np.float64), (3, 1, np.float64), (33, 3, np.float32), (100, 5, np.float32),
          (257, 2, np.float64), (1100, 2, np.float32), (600, 10, np.float32),
          (300, 16, np.float32), (70, 7, np.float64), (32, 4, np.float32),
          (1025, 3, np.float64), (130, 4, np.float32), (520, 8, np.float32),
          (400, 9, np.float32), (200, 12, np.float64), (90, 15, np.float32)]


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", LKS)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[0]}d{s[1]}{np.dtype(s[2]).name}")
def test_shapes(lk, shape, prec):
    n, d, dt = shape
    X = inputs.gaussian_mixture(n, d, 5, seed=n * 31 + d, dtype=dt)
    _assert_same(hac.cluster(X, lk, precision=prec), oracle.rounds(X.astype(np.float64), lk),
                 rtol=_rtol(lk, prec))


@pytest.mark.parametrize("lk", LKS)
def test_single_point(lk):
    got = hac.cluster(np.zeros((1, 3)), lk)
    assert len(got["a"]) == 0 and got["stats"]["rounds"] == 0


@pytest.mark.parametrize("lk", LKS)
def test_duplicates(lk):
    n = 40
    X = np.tile(np.array([[2.5, -1.0, 0.25]]), (n, 1))
    got = oracle.canonical(hac.cluster(X, lk))
    assert list(got["a"]) == [0] * (n - 1)
    assert list(got["b"]) == list(range(1, n))
    assert np.all(got["h"] == 0.0)
    assert got["stats"]["rounds"] == n - 1


@pytest.mark.parametrize("lk", LKS)
def test_huge_coordinates_take_fp64(lk):
    """FP32 point copies with a coordinate of 2^40 or more would overflow the
    FP32 paths: hac_run runs them in FP64 in either mode (same tree as the
    oracle at FP64 tolerance)."""
    rng = np.random.default_rng(77)
    X = rng.normal(size=(400, 4)) * 1e13  # extent far above 2^40 after recentring
    want = oracle.nnchain(X, lk)
    for prec in PRECS:
        got = hac.cluster(X, lk, precision=prec)
        _assert_same(got, want, rtol=RTOL64, rounds=False)
    got32 = hac.cluster(X.astype(np.float32), lk, precision=hac.PREC_F32_RECHECK)
    _assert_same(got32, oracle.nnchain(X.astype(np.float32).astype(np.float64), lk),
                 rtol=RTOL64, rounds=False)


@pytest.mark.parametrize("lk", LKS)
def test_collinear_closed_form(lk):
    m, hsp = 64, 0.25
    X = np.zeros((m, 2))
    X[:, 0] = hsp * np.arange(m)
    got = oracle.as_map(hac.cluster(X, lk))
    s = 1
    while s < m:
        for start in range(0, m, 2 * s):
            want = {"complete": (2 * s - 1) * hsp, "average": s * hsp, "ward": s ** 1.5 * hsp,
                    "average_sq": (s * hsp) ** 2 + hsp ** 2 * (s * s - 1) / 6.0}[lk]
            h, size = got[(start, start + s)]
            assert size == 2 * s and h == pytest.approx(want, rel=1e-12)
        s *= 2


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_lattice_complete_exact_ties(prec):
    for seed in range(3):
        X = inputs.lattice(500, 3, seed=seed, levels=12)
        got = hac.cluster(X, "complete", precision=prec)
        want = oracle.rounds(X.astype(np.float64), "complete")
        _assert_same(got, want, rtol=0.0 if prec == hac.PREC_F64 else RTOL32)


def _same_as_fp64(got, X, lk, **kw):
    """FP32 bulk + FP64 re-score: the tree (and the round of every merge) must
    be the all-FP64 tree's, merge for merge; heights within the FP32 bound."""
    ref = hac.cluster(X, lk, precision=hac.PREC_F64, **kw)
    _assert_same(got, ref, rtol=_rtol(lk, hac.PREC_F32_RECHECK))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", ["average", "ward", "average_sq"])
def test_lattice_ties_valid(lk, prec):
    """Exact ties: a valid greedy tree (each merge within 1e-9 of the
    smallest active distance, heights within the mode's bound), and in the
    FP32 mode the all-FP64 tree exactly."""
    X = inputs.lattice(300, 4, seed=7, levels=10)
    got = hac.cluster(X, lk, precision=prec)
    bad, stats = oracle.validate(X.astype(np.float64), lk, got, rtol=RTOL64,
                                 htol=_rtol(lk, prec))
    assert bad == 0, stats
    assert oracle.check_tree(got, len(X), rtol=_rtol(lk, prec)) == []
    if prec == hac.PREC_F32_RECHECK:
        _same_as_fp64(got, X, lk)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", LKS)
def test_multilevel_tree(lk, prec):
    """12,000 points: three tree levels, ragged last leaf and node."""
    X = inputs.gaussian_mixture(12000, 2, 40, seed=77)
    _assert_same(hac.cluster(X, lk, precision=prec), oracle.rounds(X.astype(np.float64), lk),
                 rtol=_rtol(lk, prec))


@pytest.mark.parametrize("dense", ["tree", "dense"])
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", LKS)
def test_gmm5d_sample(lk, prec, dense, monkeypatch):
    """The 5-D Gaussian-mixture workload's recipe at a size the oracle runs
    (average linkage: on the range-query search, and on the dense matrix from
    the first round)."""
    if dense == "tree":
        monkeypatch.setenv("HAC_DENSE_K", "0")
    elif lk != "average":
        pytest.skip("the dense matrix is for average linkage")
    X = inputs.workload("gmm5d_1m_f32", n=5000)
    got = hac.cluster(X, lk, precision=prec)
    _assert_same(got, oracle.rounds(X.astype(np.float64), lk), rtol=_rtol(lk, prec))
    if lk == "average":
        assert (got["stats"]["dense_k"] > 0) == (dense == "dense")


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", ["average", "ward", "average_sq"])
def test_lattice16d_sample(lk, prec):
    """The 16-D lattice tie-stress recipe at oracle size: exact ties among
    singletons break by cid identically; later near-ties are checked by the
    greedy-validity replay."""
    X = inputs.workload("lattice16d_1m_f32", n=2000)
    got = hac.cluster(X, lk, precision=prec)
    bad, stats = oracle.validate(X.astype(np.float64), lk, got, rtol=RTOL64,
                                 htol=_rtol(lk, prec))
    assert bad == 0, stats
    if prec == hac.PREC_F32_RECHECK:
        _same_as_fp64(got, X, lk)
    want = oracle.rounds(X.astype(np.float64), lk)
    # round-0 merges are between singletons at exactly representable distances
    r0 = lambda d: {(int(a), int(b)) for a, b, r in zip(d["a"], d["b"], d["round"]) if r == 0}
    assert r0(got) == r0(want)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_spreaders_sample(prec):
    X = inputs.spreaders(6000, seed=3000)
    for lk in ("ward", "complete"):
        _assert_same(hac.cluster(X, lk, precision=prec), oracle.rounds(X.astype(np.float64), lk),
                 rtol=_rtol(lk, prec))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", LKS)
def test_deterministic(lk, prec):
    X = inputs.gaussian_mixture(3000, 3, 8, seed=5)
    a, b = hac.cluster(X, lk, precision=prec), hac.cluster(X, lk, precision=prec)
    for k in ("a", "b", "size", "round"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["h"].view(np.int64), b["h"].view(np.int64))


def test_device_pointer_entry():
    torch = pytest.importorskip("torch")
    X = inputs.gaussian_mixture(2000, 4, 6, seed=9)
    t = torch.from_numpy(X).cuda()
    h = hac.hac_create_device(t.data_ptr(), X.shape[0], X.shape[1], np.float32, "ward")
    try:
        assert hac.hac_run(h) == 0
        m = hac.hac_dendrogram(h, len(X))
    finally:
        hac.hac_destroy(h)
    got = dict(a=m["cid_a"], b=m["cid_b"], h=m["height"], size=m["size"])
    _assert_same(got, oracle.nnchain(X.astype(np.float64), "ward"), rounds=False)


def test_nonfinite_device_input_rejected():
    torch = pytest.importorskip("torch")
    X = inputs.gaussian_mixture(100, 2, 3, seed=1)
    X[17, 1] = np.nan
    t = torch.from_numpy(X).cuda()
    h = hac.hac_create_device(t.data_ptr(), 100, 2, np.float32, "average")
    try:
        assert hac.hac_run(h) == hac.HAC_EINVAL
        with pytest.raises(hac.HacError):
            hac.hac_dendrogram(h, 100)
    finally:
        hac.hac_destroy(h)


def test_round_limit_and_rerun():
    X = inputs.gaussian_mixture(500, 2, 4, seed=2)
    h = hac.hac_create(X, "complete")
    try:
        assert hac.hac_run(h, max_rounds=2) == hac.HAC_ETIMEOUT
        assert hac.hac_run(h) == 0
        m = hac.hac_dendrogram(h, len(X))
        assert len(m) == len(X) - 1
    finally:
        hac.hac_destroy(h)


def test_cache_resize_between_runs(tree_path):
    """Reruns of one handle with another cache size give the same tree; a
    larger table replaces the old one (its memory is released) and a smaller
    request reuses it."""
    n = 3000
    X = inputs.gaussian_mixture(n, 3, 8, seed=21)
    want = oracle.rounds(X.astype(np.float64), "average")
    h = hac.hac_create(X, "average")
    sizes = []
    try:
        for slots in (8, 64, 16):
            assert hac.hac_run(h, precision=hac.PREC_F32_RECHECK, cache_slots=slots) == 0
            sizes.append(hac.hac_stats(h)["device_bytes"])
            m = hac.hac_dendrogram(h, n)
            got = dict(a=m["cid_a"], b=m["cid_b"], h=m["height"], size=m["size"])
            _assert_same(got, want, rtol=RTOL32, rounds=False)
    finally:
        hac.hac_destroy(h)
    cell = 8 + 8 + 4 + 4  # key, value, error term, covered part
    assert sizes[1] - sizes[0] == n * (64 - 8) * cell
    assert sizes[2] == sizes[1]


def _members_small(d, n, cap=64):
    """Members of every merged cluster of size <= cap, by replaying merges in
    size order (children before parents)."""
    mem = {}
    order = np.argsort(d["size"], kind="stable")
    out = {}
    for t in order:
        s = int(d["size"][t])
        if s > cap:
            break
        a, b = int(d["a"][t]), int(d["b"][t])
        ma = mem.pop(a, [a])
        mb = mem.pop(b, [b])
        out[t] = (ma, mb)
        mem[a] = ma + mb
    return out


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", ["ward", "average_sq"])
def test_full_size_1m_properties(lk, prec):
    """The 10^6-point 5-D workload in the benchmark's launch configuration:
    a valid tree with monotone heights, and sampled merge heights equal to the
    oracle's linkage distance of the two merged point sets."""
    X = inputs.workload("gmm5d_1m_f32")
    got = hac.cluster(X, lk, precision=prec)
    n = len(X)
    assert oracle.check_tree(got, n, rtol=1e-12) == []
    mem = _members_small(got, n)
    rng = np.random.default_rng(0)
    keys = list(mem)
    X64 = X.astype(np.float64)
    for t in rng.choice(len(keys), size=min(300, len(keys)), replace=False):
        ma, mb = mem[keys[t]]
        want = oracle.cluster_dist(lk, X64[ma], X64[mb])
        assert got["h"][keys[t]] == pytest.approx(want, rel=RTOL64, abs=1e-12)
    if lk == "ward":
        _check_rnn(got, X, lk, 24, k_big=2, every_size=True)
    else:
        _check_rnn(got, X, lk, 12, k_big=1, side_cap=512)
    if prec == hac.PREC_F64:
        _FULL[lk] = got
    else:
        # FP32 bulk + FP64 re-score must give the FP64 path's tree exactly
        ref = _FULL.get(lk) or hac.cluster(X, lk, precision=hac.PREC_F64)
        c = oracle.compare(got, ref, rtol=RTOL64)
        assert c["ok"], c


_FULL = {}
_WL = {}


def _workload(name):
    if name not in _WL:
        _WL[name] = inputs.workload(name)
    return _WL[name]


def _check_sampled(got, X, lk, rtol, k=300):
    """Sampled merges of at most 64 points: the height equals the oracle's
    Table 1 value of the two merged point sets."""
    X64 = X.astype(np.float64)
    picks = dendro.sample_small(got, k)
    assert len(picks) == k
    for t, sa, sb in picks:
        want = oracle.cluster_dist(lk, X64[sa], X64[sb])
        assert got["h"][t] == pytest.approx(want, rel=rtol, abs=1e-12), (t, len(sa), len(sb))


def _check_big(got, X, lk, rtol, k=2, max_pairs=4e8):
    """The merges with the most point pairs the oracle can afford here
    (|A| x |B| <= max_pairs): the height equals its Table 1 value of the two
    merged point sets."""
    X64 = X.astype(np.float64)
    picks = dendro.sample_big(got, k, max_pairs)
    assert len(picks) == k
    for t, sa, sb in picks:
        assert len(sa) * len(sb) > 10 ** 5  # big merges, not the small ones again
        want = oracle.cluster_dist(lk, X64[sa], X64[sb])
        assert got["h"][t] == pytest.approx(want, rel=rtol, abs=1e-12), (t, len(sa), len(sb))


def _check_rnn(got, X, lk, k_small, k_big=0, every_size=False, side_cap=None):
    """Sampled merges were reciprocal nearest neighbours among the clusters
    active in their round, every distance from the points by the oracle (for
    complete / average / avg-2 only from sides of at most side_cap points:
    the oracle's scan costs |side| x n point pairs)."""
    picks = dendro.pick_merges(got, k_small, cap=32, k_big=k_big, every_size=every_size,
                               big_cap=side_cap or 0)
    probs, ties, vals = dendro.rnn_check(got, X.astype(np.float64), lk, picks,
                                         oracle.dist_to_all, rtol=1e-9, side_cap=side_cap)
    assert probs == [], probs[:3]
    assert len(vals) == len(picks)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_full_size_1m_average(prec):
    """The benchmark's average-linkage run (10^6 points, 5-D mixture, 128
    cache slots): a valid tree, sampled heights equal to the oracle's value of
    the merged point sets, and the FP32 + FP64 re-score tree equal to the
    all-FP64 tree, merge for merge and round for round."""
    X = _workload("gmm5d_1m_f32")
    got = hac.cluster(X, "average", precision=prec, cache_slots=128)
    rtol = _rtol("average", prec)
    assert dendro.check(got, len(X), rtol=2 * rtol) == []
    _check_sampled(got, X, "average", rtol)
    _check_big(got, X, "average", rtol)
    _check_rnn(got, X, "average", 12, k_big=1, side_cap=512)
    if prec == hac.PREC_F64:
        _FULL["average"] = got
    else:
        ref = _FULL.get("average") or hac.cluster(X, "average", precision=hac.PREC_F64,
                                                  cache_slots=128)
        c = oracle.compare(got, ref, rtol=RTOL32)
        assert c["ok"], c
        assert _round_sets(got) == _round_sets(ref)


@pytest.mark.parametrize("lk", ["ward", "complete"])
def test_full_size_10m_spreaders(lk):
    """The 10^7-point 2-D spreader workload as one instance (FP32 + FP64
    re-score, 128 cache slots for complete): a valid tree and sampled heights
    equal to the oracle's value of the merged point sets."""
    X = _workload("spread2d_10m_f32")
    got = hac.cluster(X, lk, precision=hac.PREC_F32_RECHECK,
                      cache_slots=0 if lk == "ward" else 128)
    rtol = _rtol(lk, hac.PREC_F32_RECHECK)
    assert dendro.check(got, len(X), rtol=2 * rtol) == []
    _check_sampled(got, X, lk, rtol)
    if lk == "ward":
        _check_rnn(got, X, lk, 8, k_big=2, every_size=True)
    else:
        _check_rnn(got, X, lk, 6, side_cap=32)


@pytest.mark.parametrize("lk", ["ward", "average", "average_sq"])
def test_full_size_16d_lattice(lk):
    """The 10^6-point 16-D lattice (exact ties everywhere) with the FP32 bulk
    and the exhaustive scans of d > 8 (average linkage: candidate lists, then
    the dense matrix; 128 cache slots): a valid tree, sampled heights equal
    to the oracle's value of the merged point sets, sampled merges of
    reciprocal nearest neighbours, and for Ward and average the all-FP64
    GPU tree merge for merge and round for round (runs stop at 10 minutes
    rather than hold the GPU)."""
    X = _workload("lattice16d_1m_f32")
    slots = 128 if lk == "average" else 0
    got = hac.cluster(X, lk, precision=hac.PREC_F32_RECHECK, cache_slots=slots, timeout_s=600.0)
    rtol = _rtol(lk, hac.PREC_F32_RECHECK)
    assert dendro.check(got, len(X), rtol=2 * rtol) == []
    _check_sampled(got, X, lk, rtol)
    if lk == "ward":
        _check_rnn(got, X, lk, 20, k_big=2, every_size=True)
    else:
        _check_rnn(got, X, lk, 8, side_cap=32)
    if lk != "average_sq":
        ref = hac.cluster(X, lk, precision=hac.PREC_F64, cache_slots=slots, timeout_s=600.0)
        _assert_same(got, ref, rtol=rtol)


@pytest.mark.parametrize("slots", [8, 64])
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", ["complete", "average"])
def test_cache_parity(lk, prec, slots, tree_path):
    """Section 5 cache with the Lance-Williams update after merges: the tree
    is unchanged, heights stay within 1e-9 of the oracle, and the cache is
    actually used (hits and Lance-Williams-derived entries)."""
    X = inputs.workload("gmm5d_1m_f32", n=6000)
    got = hac.cluster(X, lk, precision=prec, cache_slots=slots)
    _assert_same(got, oracle.rounds(X.astype(np.float64), lk), rtol=_rtol(lk, prec))
    assert got["stats"]["cache_hits"] > 0 and got["stats"]["cache_lw_entries"] > 0


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", ["complete", "average"])
def test_cache_lattice_ties(lk, prec, tree_path):
    X = inputs.lattice(400, 3, seed=11, levels=16)
    got = hac.cluster(X, lk, precision=prec, cache_slots=64)
    bad, stats = oracle.validate(X.astype(np.float64), lk, got, rtol=RTOL64,
                                 htol=_rtol(lk, prec))
    assert bad == 0, stats
    if lk == "complete":  # max of exact values: Lance-Williams is exact too
        _assert_same(got, oracle.rounds(X.astype(np.float64), lk),
                     rtol=0.0 if prec == hac.PREC_F64 else RTOL32)
    if prec == hac.PREC_F32_RECHECK:
        _same_as_fp64(got, X, lk, cache_slots=64)


@pytest.mark.parametrize("slots", [8, 64])
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("lk", ["complete", "average"])
def test_big_pair_deferral(lk, prec, slots, monkeypatch, tree_path):
    """Force nearly every cached pair through the GPU-wide evaluation and
    the re-run search (tiny thresholds): the tree must not change."""
    monkeypatch.setenv("HAC_BIG_PAIRS", "256")
    monkeypatch.setenv("HAC_BIG_PAIRS_F64", "128")
    for seed, n in ((1, 3000), (2, 5000)):
        X = inputs.gaussian_mixture(n, 4, 10, seed=seed)
        got = hac.cluster(X, lk, precision=prec, cache_slots=slots)
        _assert_same(got, oracle.rounds(X.astype(np.float64), lk), rtol=_rtol(lk, prec))


@pytest.mark.parametrize("lk", ["complete", "average"])
@pytest.mark.parametrize("d", list(range(1, 17)))
def test_big_pairs_every_dimension(lk, d, monkeypatch, tree_path):
    """The GPU-wide FP32 kernels are specialised on the true dimension and
    the FP64 ones on the padded width: with tiny thresholds nearly every
    evaluated pair of >= 256 point pairs goes through them, at every d from 1
    to 16 (pairs up to ~2,100 x 1,100 points), FP32 with the FP64 re-score,
    and all-FP64 at d = 3 and 12 (padded widths 4 and 16)."""
    monkeypatch.setenv("HAC_BIG_PAIRS", "256")
    monkeypatch.setenv("HAC_BIG_PAIRS_F64", "128")
    X = inputs.gaussian_mixture(3200, d, 3, seed=100 + d,
                                dtype=np.float64 if d == 1 else np.float32)
    want = oracle.rounds(X.astype(np.float64), lk)
    for prec in [hac.PREC_F32_RECHECK] + ([hac.PREC_F64] if d in (3, 12) else []):
        got = hac.cluster(X, lk, precision=prec, cache_slots=8)
        _assert_same(got, want, rtol=_rtol(lk, prec))
        assert got["stats"]["big_point_pairs"] > 0


_PAPER_ORACLE = {}


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("name", ["uniformfill2d_1m_f32", "gaussiandisc2d_1m_f32",
                                  "uniformfill5d_1m_f32", "gaussiandisc5d_1m_f32"])
def test_paper_shapes_sample(name, prec):
    """The paper's UniformFill / GaussianDisc shapes at oracle size, every
    linkage (the cache on for complete and average, as the bench runs them)."""
    X = inputs.workload(name, n=3000)
    X64 = X.astype(np.float64)
    for lk in LKS:
        key = (name, lk)
        if key not in _PAPER_ORACLE:
            _PAPER_ORACLE[key] = oracle.rounds(X64, lk)
        slots = 64 if lk in ("complete", "average") else 0
        _assert_same(hac.cluster(X, lk, precision=prec, cache_slots=slots), _PAPER_ORACLE[key],
                     rtol=_rtol(lk, prec))


@pytest.mark.parametrize("lk", LKS)
def test_no_prune_ablation_same_tree(lk, tree_path):
    """HAC_FLAG_NO_PRUNE makes every cluster a candidate: the same tree, and
    the range query is what keeps the evaluations far below the naive count
    (average linkage on the range-query search, not the dense matrix)."""
    X = inputs.workload("gaussiandisc2d_1m_f32", n=2500)
    slots = 64 if lk in ("complete", "average") else 0
    a = hac.cluster(X, lk, precision=hac.PREC_F32_RECHECK, cache_slots=slots)
    b = hac.cluster(X, lk, precision=hac.PREC_F32_RECHECK, cache_slots=slots, no_prune=True)
    want = oracle.rounds(X.astype(np.float64), lk)
    _assert_same(a, want, rtol=_rtol(lk, hac.PREC_F32_RECHECK))
    _assert_same(b, want, rtol=_rtol(lk, hac.PREC_F32_RECHECK))
    naive = a["stats"]["naive_pairs"]
    assert naive == b["stats"]["naive_pairs"] > 0
    assert b["stats"]["leaf_tests"] >= a["stats"]["leaf_tests"]
    assert a["stats"]["cluster_pairs"] < 0.2 * naive


@pytest.mark.parametrize("lk", ["ward", "average_sq"])
@pytest.mark.parametrize("shape", [(4000, 5), (3000, 10), (2500, 16)], ids=lambda s: f"n{s[0]}d{s[1]}")
def test_exhaustive_search_matches(lk, shape, monkeypatch):
    """The tiled exhaustive search (on by default for d > 8 in the FP32 mode,
    forced here for d = 5 too) gives the oracle's tree."""
    monkeypatch.setenv("HAC_BRUTE", "1")
    n, d = shape
    X = inputs.gaussian_mixture(n, d, 7, seed=n + d)
    got = hac.cluster(X, lk, precision=hac.PREC_F32_RECHECK)
    _assert_same(got, oracle.rounds(X.astype(np.float64), lk), rtol=RTOL64)
    st = got["stats"]
    assert st["nodes_visited"] == 0          # no tree traversal
    assert st["leaf_tests"] >= st["naive_pairs"]  # every cluster scanned per terminal
