"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check is a worked example
(Fig. 1), a closed form, a textbook special case, an independent brute-force
algorithm that recomputes distances from the points, or an invariant the
paper proves.  ``test_pins_catch_mutants`` shows the pins are sensitive by
planting plausible mistakes in a copy of the oracle source.
"""
import itertools
import json
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2106_04727_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LKS = ["complete", "average", "ward", "average_sq"]


def _fig1():
    with open(os.path.join(GOLDEN, "fig1_six_points.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Worked example: Fig. 1 / Section 1
# ---------------------------------------------------------------------------

def test_fig1_round_structure():
    g = _fig1()
    X = np.array(g["points"], dtype=np.float64)
    r = oracle.rounds(X, g["linkage"], log_terminals=True)
    assert r["n_rounds"] == g["n_rounds"]
    got = {}
    for a, b, rr in zip(r["a"], r["b"], r["round"]):
        got.setdefault(int(rr), set()).add((int(a), int(b)))
    want = {i: {tuple(p) for p in ms} for i, ms in enumerate(g["round_merges"])}
    assert got == want
    terms = {}
    for rr, c in r["terminals"]:
        terms.setdefault(int(rr), set()).add(int(c))
    assert terms == {i: set(t) for i, t in enumerate(g["round_terminals"])}
    # f (index 5) does no search in round 2 (index 1)
    assert 5 not in terms[1]


def test_fig1_heights_and_chain():
    g = _fig1()
    X = np.array(g["points"], dtype=np.float64)
    for fn in (oracle.nnchain, oracle.rounds, oracle.greedy):
        d = fn(X, g["linkage"])
        m = oracle.as_map(d)
        assert set(m) == {tuple(map(int, k.split(","))) for k in g["squared_heights"]}
        for k, h2 in g["squared_heights"].items():
            key = tuple(map(int, k.split(",")))
            assert m[key][0] == math.sqrt(h2)  # exact: integer coordinates
    # first-round successors from brute-force point NN with the (d, cid) key
    D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    for i, j in g["first_round_successor"].items():
        i = int(i)
        best = min(range(6), key=lambda t: (D[i, t], t))
        assert best == j


# ---------------------------------------------------------------------------
# Closed forms and special cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lk", LKS)
def test_two_points(lk):
    X = np.array([[0.5, -1.0, 2.0], [3.5, 3.0, 2.0]])
    for fn in (oracle.nnchain, oracle.rounds, oracle.greedy):
        d = fn(X, lk)
        assert list(d["a"]) == [0] and list(d["b"]) == [1] and list(d["size"]) == [2]
        # avg-2 is the mean SQUARED distance (Table 1)
        assert d["h"][0] == pytest.approx(25.0 if lk == "average_sq" else 5.0, rel=1e-15)


@pytest.mark.parametrize("lk", LKS)
def test_single_point(lk):
    d = oracle.nnchain(np.zeros((1, 2)), lk)
    assert len(d["a"]) == 0


@pytest.mark.parametrize("lk", LKS)
def test_collinear_equally_spaced(lk):
    """16 points 0, h, 2h, ...: ties everywhere; the (D, cid) key merges
    neighbours pairwise, then pairs of pairs, ... (a balanced tree).  Merging
    two blocks of s points at centroid spacing s*h gives complete (2s-1)h,
    average s*h, Ward sqrt(2 s^2/(2s) (s h)^2) = s^1.5 h and avg-2
    (s h)^2 + 2 h^2 (s^2 - 1)/12 (squared centroid gap plus both blocks'
    per-point variances)."""
    m, hsp = 16, 0.5
    X = np.zeros((m, 3))
    X[:, 1] = hsp * np.arange(m)
    want = {}
    s = 1
    while s < m:
        for start in range(0, m, 2 * s):
            if lk == "complete":
                h = (2 * s - 1) * hsp
            elif lk == "average":
                h = s * hsp
            elif lk == "ward":
                h = s ** 1.5 * hsp
            else:
                h = (s * hsp) ** 2 + hsp ** 2 * (s * s - 1) / 6.0
            want[(start, start + s)] = (h, 2 * s)
        s *= 2
    for fn in (oracle.nnchain, oracle.rounds, oracle.greedy):
        got = oracle.as_map(fn(X, lk))
        assert set(got) == set(want), fn.__name__
        for k in want:
            assert got[k][1] == want[k][1]
            assert got[k][0] == pytest.approx(want[k][0], rel=1e-13)


@pytest.mark.parametrize("lk", LKS)
def test_all_duplicates(lk):
    """All points equal: every height is 0 and the key (0, min cid, max cid)
    always picks cluster 0 with the next index."""
    n = 9
    X = np.tile([[1.25, -3.0]], (n, 1))
    for fn in (oracle.nnchain, oracle.rounds, oracle.greedy):
        d = oracle.canonical(fn(X, lk))
        assert list(d["a"]) == [0] * (n - 1)
        assert list(d["b"]) == list(range(1, n))
        assert list(d["size"]) == list(range(2, n + 1))
        assert np.all(d["h"] == 0.0)
    r = oracle.rounds(X, lk)
    assert r["n_rounds"] == n - 1   # one merge per round on a full tie


def test_ward_singletons_are_euclidean():
    rng = np.random.default_rng(5)
    A, B = rng.normal(size=(1, 4)), rng.normal(size=(1, 4))
    assert oracle.cluster_dist("ward", A, B) == pytest.approx(np.linalg.norm(A - B), rel=1e-15)


def test_ward_closed_form_variance_increase():
    """Table 1: Ward = sqrt(2 (Var(A u B) - Var(A) - Var(B)))."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        A = rng.normal(size=(rng.integers(1, 9), 3))
        B = rng.normal(size=(rng.integers(1, 9), 3)) + 2.0
        var = lambda P: ((P - P.mean(0)) ** 2).sum()
        want = math.sqrt(2 * (var(np.vstack([A, B])) - var(A) - var(B)))
        assert oracle.cluster_dist("ward", A, B) == pytest.approx(want, rel=1e-11)


@pytest.mark.parametrize("lk", LKS)
def test_lance_williams_matches_definition(lk):
    """Table 2 update of D(A u B, C) equals the Table 1 definition recomputed
    from the points (squared distances for Ward)."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        A, B, C = (rng.normal(size=(rng.integers(1, 7), 2)) * rng.uniform(0.1, 3)
                   + rng.normal(size=2) * 3 for _ in range(3))
        f = (lambda P, Q: oracle.cluster_dist(lk, P, Q) ** 2) if lk == "ward" else \
            (lambda P, Q: oracle.cluster_dist(lk, P, Q))
        got = oracle.lw(lk, f(A, C), f(B, C), f(A, B), len(A), len(B), len(C))
        want = f(np.vstack([A, B]), C)
        assert got == pytest.approx(want, rel=1e-11, abs=1e-12)


def test_lance_williams_complete_coefficients():
    """a1 = a2 = c = 1/2, b = 0 reproduces the max."""
    for x, y in [(1.0, 2.0), (3.0, 0.5), (2.0, 2.0)]:
        lw = 0.5 * x + 0.5 * y + 0.5 * abs(x - y)
        assert oracle.lw("complete", x, y, 7.0, 3, 4, 5) == lw == max(x, y)


def test_avg2_closed_form():
    """Table 1: the mean squared distance between A and B equals the squared
    centroid gap plus both clusters' per-point variances (computed here from
    the points with numpy, not by the oracle)."""
    rng = np.random.default_rng(16)
    for _ in range(40):
        A = rng.normal(size=(rng.integers(1, 9), 3)) * rng.uniform(0.2, 2)
        B = rng.normal(size=(rng.integers(1, 9), 3)) + rng.normal(size=3) * 2
        pv = lambda P: ((P - P.mean(0)) ** 2).sum(1).mean()
        want = ((A.mean(0) - B.mean(0)) ** 2).sum() + pv(A) + pv(B)
        assert oracle.cluster_dist("average_sq", A, B) == pytest.approx(want, rel=1e-12)
        brute = np.mean([((x - y) ** 2).sum() for x in A for y in B])
        assert oracle.cluster_dist("average_sq", A, B) == pytest.approx(brute, rel=1e-13)


@pytest.mark.parametrize("lk", LKS)
def test_dist_to_all_matches_library_and_variance_forms(lk):
    """The linear-memory distance from one cluster of a labelling to all
    others: mean / max / mean square of scipy's point-distance matrix, and for
    Ward the variance-increase form sqrt(2 (SSE(Q u C) - SSE(Q) - SSE(C)))
    computed with numpy; NaN for the query itself and for unused labels."""
    cdist = pytest.importorskip("scipy.spatial.distance").cdist
    rng = np.random.default_rng(23)
    X = rng.normal(size=(90, 3)) * rng.uniform(0.5, 2, size=3)
    label = rng.integers(0, 9, size=90) * 2  # odd labels unused
    label[:9] = np.arange(9) * 2
    sse = lambda P: ((P - P.mean(0)) ** 2).sum()
    for q in (0, 6, 16):
        got = oracle.dist_to_all(lk, X, label, q)
        Q = X[label == q]
        assert len(got) == 17 and math.isnan(got[q])
        for c in range(17):
            C = X[label == c]
            if c == q or not len(C):
                assert math.isnan(got[c])
                continue
            M = cdist(Q, C)
            want = {"complete": M.max(), "average": M.mean(), "average_sq": (M ** 2).mean(),
                    "ward": math.sqrt(2 * (sse(np.vstack([Q, C])) - sse(Q) - sse(C)))}[lk]
            assert got[c] == pytest.approx(want, rel=1e-11)


def test_centroid_lower_bound():
    """Section 4.2 proof: ||c_A - c_B|| <= D_avg(A,B) <= D_comp(A,B)."""
    rng = np.random.default_rng(8)
    for _ in range(100):
        A = rng.normal(size=(rng.integers(1, 12), 3))
        B = rng.normal(size=(rng.integers(1, 12), 3)) + rng.normal(size=3)
        c = np.linalg.norm(A.mean(0) - B.mean(0))
        avg = oracle.cluster_dist("average", A, B)
        comp = oracle.cluster_dist("complete", A, B)
        assert c <= avg * (1 + 1e-12) and avg <= comp * (1 + 1e-12)


def test_summary_upper_bounds():
    """The summary upper bounds the search offers before evaluating a pair
    (no point pairs needed): D_avg(A,B) <= sqrt(||c_A - c_B||^2 + var A +
    var B) with per-point variances (Jensen: the mean of ||x - y|| is at most
    the root of the mean of ||x - y||^2, which is that sum), and D_comp(A,B)
    at most the distance between the farthest corners of the two bounding
    boxes; both reach equality for singletons."""
    rng = np.random.default_rng(10)
    for _ in range(200):
        d = int(rng.integers(1, 6))
        A = rng.normal(size=(rng.integers(1, 12), d)) * rng.uniform(0.1, 3)
        B = rng.normal(size=(rng.integers(1, 12), d)) * rng.uniform(0.1, 3) + rng.normal(size=d) * 3
        pv = lambda P: ((P - P.mean(0)) ** 2).sum(1).mean()
        ub_avg = math.sqrt(((A.mean(0) - B.mean(0)) ** 2).sum() + pv(A) + pv(B))
        far = np.maximum(np.abs(A.max(0) - B.min(0)), np.abs(B.max(0) - A.min(0)))
        ub_comp = math.sqrt((far ** 2).sum())
        assert oracle.cluster_dist("average", A, B) <= ub_avg * (1 + 1e-12)
        assert oracle.cluster_dist("complete", A, B) <= ub_comp * (1 + 1e-12)
    x, y = rng.normal(size=(1, 3)), rng.normal(size=(1, 3))
    assert oracle.cluster_dist("average", x, y) == pytest.approx(np.linalg.norm(x - y), rel=1e-14)
    far = np.abs(x - y)
    assert oracle.cluster_dist("complete", x, y) == pytest.approx(np.linalg.norm(far), rel=1e-14)


def test_complete_linkage_necessary_conditions():
    """Section 4.3 reading: the search keeps a candidate B for complete
    linkage only if ||c_i - c_B|| <= beta and, on every axis,
    max(hi_B - lo_A, hi_A - lo_B) <= beta; both are implied by
    D_comp(A, B) <= beta (every point pair is within D_comp, on every axis)."""
    rng = np.random.default_rng(12)
    for _ in range(300):
        d = int(rng.integers(1, 5))
        A = rng.normal(size=(rng.integers(1, 10), d))
        B = rng.normal(size=(rng.integers(1, 10), d)) + rng.normal(size=d)
        beta = oracle.cluster_dist("complete", A, B) * rng.uniform(1.0, 1.3)
        assert np.linalg.norm(A.mean(0) - B.mean(0)) <= beta * (1 + 1e-12)
        ext = np.maximum(B.max(0) - A.min(0), A.max(0) - B.min(0))
        assert np.all(ext <= beta * (1 + 1e-12))


def test_ward_radius_soundness():
    """Section 4.1: if Ward(Ci, B) <= beta then ||c_i - c_B|| <= beta *
    sqrt((|Ci| + n_min) / (2 n_min |Ci|)) for any |B| >= n_min."""
    rng = np.random.default_rng(9)
    for _ in range(200):
        A = rng.normal(size=(rng.integers(1, 10), 2))
        B = rng.normal(size=(rng.integers(1, 10), 2)) * 0.5 + rng.normal(size=2)
        nmin = rng.integers(1, len(B) + 1)
        beta = oracle.cluster_dist("ward", A, B) * rng.uniform(1.0, 1.5)
        r = beta * math.sqrt((len(A) + nmin) / (2.0 * nmin * len(A)))
        assert np.linalg.norm(A.mean(0) - B.mean(0)) <= r * (1 + 1e-12)


# ---------------------------------------------------------------------------
# Independent brute force and invariants
# ---------------------------------------------------------------------------

def _random_sets():
    for seed in range(6):
        n = [2, 3, 7, 23, 64, 97][seed]
        yield f"uniform{n}", inputs.uniform_cube(n, 2, seed=100 + seed)
        yield f"gmm{n}", inputs.gaussian_mixture(n, 3, 4, seed=200 + seed).astype(np.float64)


@pytest.mark.parametrize("lk", LKS)
def test_nnchain_equals_bruteforce(lk):
    for name, X in _random_sets():
        want = oracle.greedy(X, lk)
        for fn in (oracle.nnchain, oracle.rounds):
            got = fn(X, lk)
            c = oracle.compare(got, want, rtol=1e-12)
            assert c["ok"], (name, fn.__name__, c)
            assert oracle.check_tree(got, len(X)) == []


@pytest.mark.parametrize("lk", LKS)
def test_start_independence(lk):
    X = inputs.gaussian_mixture(150, 2, 5, seed=11).astype(np.float64)
    base = oracle.nnchain(X, lk, start=0)
    for st in (1, 37, 149):
        c = oracle.compare(oracle.nnchain(X, lk, start=st), base, rtol=1e-12)
        assert c["same_tree"], (st, c)


@pytest.mark.parametrize("lk", LKS)
def test_unit_square_exact_ties(lk):
    """Four corners of the unit square, every singleton nearest-neighbour
    distance tied at 1 (hand-derived).  Round 0: 0 -> {1, 2} picks 1 (smaller
    cid), 1 -> {0, 3} picks 0, 2 -> {0, 3} picks 0, 3 -> {1, 2} picks 1; only
    {0, 1} is reciprocal.  Round 1: the pair {2, 3} at 1 is closer than either
    to {0, 1}.  Round 2: the two sides.  Breaking ties toward the larger cid
    would instead merge {0, 2} and {1, 3} in round 0."""
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    r2 = math.sqrt(2.0)
    top = {"complete": r2, "average": (1 + r2) / 2, "ward": r2, "average_sq": 1.5}[lk]
    got = oracle.rounds(X, lk)
    rec = sorted(zip(got["round"].tolist(), got["a"].tolist(), got["b"].tolist(),
                     got["size"].tolist(), got["h"].tolist()))
    want = [(0, 0, 1, 2, 1.0), (1, 2, 3, 2, 1.0), (2, 0, 2, 4, top)]
    assert [r[:4] for r in rec] == [w[:4] for w in want]
    for r, w in zip(rec, want):
        assert r[4] == pytest.approx(w[4], rel=1e-15)


def test_lattice_complete_exact_ties():
    """On a coarse lattice every complete-linkage value is sqrt of an exact
    FP64 integer multiple of the step^2, so ties are exact and the Lance-
    Williams matrix and the brute force must agree merge for merge."""
    for seed in range(4):
        X = inputs.lattice(60, 3, seed=seed, levels=6).astype(np.float64)
        want = oracle.greedy(X, "complete")
        for fn in (oracle.nnchain, oracle.rounds):
            c = oracle.compare(fn(X, "complete"), want, rtol=0.0)
            assert c["ok"], (seed, fn.__name__, c)


@pytest.mark.parametrize("lk", ["average", "ward", "average_sq"])
def test_lattice_ties_validate(lk):
    """With exact real ties, average/Ward values from different rounding
    orders may break ties differently (and a different early choice changes
    later heights); both trees must still be valid greedy dendrograms."""
    for seed in range(3):
        X = inputs.lattice(50, 3, seed=seed, levels=5).astype(np.float64)
        a, b = oracle.nnchain(X, lk), oracle.greedy(X, lk)
        for d in (a, b):
            bad, stats = oracle.validate(X, lk, d, rtol=1e-9)
            assert bad == 0, (seed, stats)


@pytest.mark.parametrize("lk", LKS)
def test_validate_detects_planted_errors(lk):
    X = inputs.uniform_cube(40, 2, seed=3)
    d = oracle.nnchain(X, lk)
    assert oracle.validate(X, lk, d)[0] == 0
    bad = {k: v.copy() for k, v in d.items()}
    i = int(np.argmax(bad["h"] > np.median(bad["h"])))
    bad["h"][i] *= 1.01
    assert oracle.validate(X, lk, bad)[0] != 0
    # a tree built for another linkage is (generically) not valid for this one
    other = oracle.nnchain(X, {"complete": "ward", "average": "complete", "ward": "average",
                               "average_sq": "complete"}[lk])
    assert oracle.validate(X, lk, other)[0] != 0


@pytest.mark.parametrize("lk", LKS)
def test_validate_tolerances_are_separate(lk):
    """The replay's two tolerances act on different things: `htol` on the
    reported heights only, `rtol` on how far a merge may sit above the
    smallest active distance.  Planted: every height 5e-6 too high (a valid
    tree), and a tree whose first merge is 1e-7 (relative) above the minimum
    with exact heights."""
    X = inputs.uniform_cube(40, 2, seed=5)
    d = oracle.nnchain(X, lk)
    hi = dict(d, h=d["h"] * (1 + 5e-6))
    assert oracle.validate(X, lk, hi, rtol=1e-9, htol=1e-5)[0] == 0
    assert oracle.validate(X, lk, hi, rtol=1e-9, htol=1e-6)[0] != 0
    assert oracle.validate(X, lk, hi, rtol=1e-5, htol=1e-6)[0] != 0
    # 1-D points 0, 1, 2 + 1e-7: merging {1, 2} first is not the minimum
    P = np.array([[0.0], [1.0], [2.0 + 1e-7]])
    h1 = oracle.cluster_dist(lk, P[[1]], P[[2]])
    h2 = oracle.cluster_dist(lk, P[[0]], P[[1, 2]])
    planted = dict(a=np.array([1, 0]), b=np.array([2, 1]), h=np.array([h1, h2]),
                   size=np.array([2, 3]))
    bad, stats = oracle.validate(P, lk, planted, rtol=1e-9, htol=1.0)
    assert bad == 1 and 1e-8 < stats[1] < 1e-6, stats
    bad, stats = oracle.validate(P, lk, planted, rtol=1e-6, htol=1e-12)
    assert bad == 0 and stats[0] == 1, stats


@pytest.mark.parametrize("lk", LKS)
def test_rounds_monotone_and_tree(lk):
    X = inputs.gaussian_mixture(300, 2, 6, seed=21).astype(np.float64)
    r = oracle.rounds(X, lk)
    assert oracle.check_tree(r, len(X)) == []
    assert r["round"].max() == r["n_rounds"] - 1
    # per round, merged clusters are disjoint (each cid appears at most once)
    for rr in range(r["n_rounds"]):
        sel = r["round"] == rr
        ids = np.concatenate([r["a"][sel], r["b"][sel]])
        assert len(ids) == len(set(ids.tolist())) and sel.sum() >= 1


def test_scipy_crosscheck():
    """scipy's NN-chain / generic implementations (run, not copied) as a
    third-party check on heights and tree for all three linkages."""
    sch = pytest.importorskip("scipy.cluster.hierarchy")
    X = inputs.gaussian_mixture(200, 3, 5, seed=31).astype(np.float64)
    n = len(X)
    from scipy.spatial.distance import pdist
    for lk in LKS:
        if lk == "average_sq":  # average linkage on squared Euclidean distances
            Z = sch.linkage(pdist(X, "sqeuclidean"), method="average")
        else:
            Z = sch.linkage(X, method=lk)
        cid = list(range(n))
        m = {}
        for i, (p, q, h, cnt) in enumerate(Z):
            a, b = cid[int(p)], cid[int(q)]
            m[(min(a, b), max(a, b))] = (float(h), int(cnt))
            cid.append(min(a, b))
        got = oracle.as_map(oracle.nnchain(X, lk))
        assert set(got) == set(m), lk
        for k in m:
            assert got[k][1] == m[k][1]
            assert got[k][0] == pytest.approx(m[k][0], rel=1e-10)


# ---------------------------------------------------------------------------
# Mutation check: plausible oracle mistakes are caught by the pins above
# ---------------------------------------------------------------------------

MUTANTS = {
    "ward_b_sign": ("- nc * dab) / (na + nb + nc)", "+ nc * dab) / (na + nb + nc)"),
    "ward_a1_uses_nb": ("return ((na + nc) * dac", "return ((nb + nc) * dac"),
    "avg_weights_swapped": ("return (na * dac + nb * dbc) / (na + nb);",
                            "return (nb * dac + na * dbc) / (na + nb);"),
    "complete_min": ("return fmax(dac, dbc);", "return fmin(dac, dbc);"),
    "tie_prefers_larger_cid": ("if (best < 0 || v < bd) {", "if (best < 0 || v <= bd) {"),
    "ward_not_squared": ("if (linkage == LK_WARD || linkage == LK_AVG2)",
                         "if (linkage == LK_AVG2)"),
    "avg2_not_squared": ("if (linkage == LK_WARD || linkage == LK_AVG2)",
                         "if (linkage == LK_WARD)"),
}


@pytest.mark.parametrize("mut", sorted(MUTANTS))
def test_pins_catch_mutants(mut, tmp_path):
    import ctypes
    src = open(os.path.join(os.path.dirname(oracle.__file__), "hac_oracle.c")).read()
    old, new = MUTANTS[mut]
    assert src.count(old) == 1
    path = tmp_path / "m.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "m.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_nnchain.argtypes = [P, i64, ctypes.c_int, ctypes.c_int, i64, P, P, P, P]
    caught = False
    cases = list(_random_sets()) + [("dups", np.tile([[0.0, 1.0]], (5, 1))),
                                    ("collinear", np.c_[np.arange(8.0), np.zeros(8)])]
    for lk, (name, X) in itertools.product(range(4), cases):
        X = np.ascontiguousarray(X, dtype=np.float64)
        n = len(X)
        a, b, h, s = (np.zeros(n - 1, np.int64), np.zeros(n - 1, np.int64),
                      np.zeros(n - 1), np.zeros(n - 1, np.int64))
        p = lambda v: v.ctypes.data_as(P)
        lib.oracle_nnchain(p(X), n, X.shape[1], lk, 0, p(a), p(b), p(h), p(s))
        got = dict(a=a, b=b, h=h, size=s)
        if not oracle.compare(got, oracle.greedy(X, lk), rtol=1e-9)["ok"]:
            caught = True
            break
    assert caught, mut


DIST_MUTANTS = {
    "avg_mean_over_one_side": ("else out[c] = acc[c] / ((double)nq * (double)cnt[c]);",
                               "else out[c] = acc[c] / (double)cnt[c];"),
    "complete_min": ("if (v > acc[c]) acc[c] = v;", "if (v < acc[c] || acc[c] == 0.0) acc[c] = v;"),
    "avg2_unsquared": ("acc[c] += point_dist2(x, y, d);", "acc[c] += point_dist(x, y, d);"),
    "ward_no_two": ("out[c] = sqrt(2.0 * (double)nq * (double)cnt[c] / (double)(nq + cnt[c]) * dd);",
                    "out[c] = sqrt((double)nq * (double)cnt[c] / (double)(nq + cnt[c]) * dd);"),
    "ward_query_sum_not_mean": ("for (int k = 0; k < d; ++k) mq[k] /= (double)nq;", ""),
}


@pytest.mark.parametrize("mut", sorted(DIST_MUTANTS))
def test_dist_to_all_pin_catches_mutants(mut, tmp_path):
    """The library-based pin of oracle_dist_to_all rejects plausible mistakes
    planted in a copy of the oracle source."""
    import ctypes
    cdist = pytest.importorskip("scipy.spatial.distance").cdist
    src = open(os.path.join(os.path.dirname(oracle.__file__), "hac_oracle.c")).read()
    old, new = DIST_MUTANTS[mut]
    assert src.count(old) == 1
    path = tmp_path / "m.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "m.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.oracle_dist_to_all.argtypes = [i32, P, i64, i32, P, i64, i64, P]
    rng = np.random.default_rng(29)
    X = np.ascontiguousarray(rng.normal(size=(60, 3)) * 2.0)
    label = np.ascontiguousarray(rng.integers(0, 5, size=60), dtype=np.int64)
    label[:5] = np.arange(5)
    sse = lambda Q: ((Q - Q.mean(0)) ** 2).sum()
    caught = False
    for lk, q in itertools.product(range(4), range(5)):
        out = np.empty(5)
        lib.oracle_dist_to_all(lk, X.ctypes.data_as(P), 60, 3, label.ctypes.data_as(P), 5, q,
                               out.ctypes.data_as(P))
        Q = X[label == q]
        for c in range(5):
            if c == q:
                continue
            C = X[label == c]
            M = cdist(Q, C)
            want = [M.max(), M.mean(), math.sqrt(2 * (sse(np.vstack([Q, C])) - sse(Q) - sse(C))),
                    (M ** 2).mean()][lk]
            if not abs(out[c] - want) <= 1e-11 * abs(want):
                caught = True
    assert caught, mut
