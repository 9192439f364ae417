"""GPU parity of the dense phase of average linkage (the full matrix of
cluster-pair distances once the active clusters fit, filled by one all-pairs
sweep and updated by Lance-Williams): against the CPU oracle merge for merge
and round for round, from the first round and after a switch in mid-run, with
exact ties, in both precision modes; the sweep's point-pair count is the exact
number of pairs in different clusters."""
import numpy as np
import pytest

import oracle
from paper_2106_04727_gb300 import hac, inputs

pytestmark = pytest.mark.gpu

PRECS = [hac.PREC_F64, hac.PREC_F32_RECHECK]
PREC_IDS = ["f64", "f32recheck"]


def _rtol(prec):
    return 1e-9 if prec == hac.PREC_F64 else 1e-5


def _round_sets(d):
    out = {}
    for a, b, r in zip(d["a"], d["b"], d["round"]):
        out.setdefault(int(r), set()).add((int(a), int(b)))
    return out


def _same(got, want, rtol):
    c = oracle.compare(got, want, rtol=rtol)
    assert c["ok"], c
    assert _round_sets(got) == _round_sets(want)


SHAPES = [(2, 2, np.float64), (3, 1, np.float64), (33, 3, np.float32), (100, 5, np.float32),
          (257, 2, np.float64), (1100, 2, np.float32), (600, 10, np.float32),
          (300, 16, np.float32), (70, 7, np.float64), (1025, 3, np.float64),
          (520, 8, np.float32), (400, 9, np.float32), (200, 12, np.float64), (90, 15, np.float32),
          (2100, 4, np.float32), (1500, 16, np.float64)]


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[0]}d{s[1]}{np.dtype(s[2]).name}")
def test_dense_from_first_round(shape, prec, monkeypatch):
    """n below the switch size: every round runs on the matrix; the sweep
    visits each of the n(n-1)/2 point pairs exactly once."""
    monkeypatch.setenv("HAC_DENSE_K", "65536")
    n, d, dt = shape
    X = inputs.gaussian_mixture(n, d, 5, seed=n * 17 + d, dtype=dt)
    got = hac.cluster(X, "average", precision=prec)
    _same(got, oracle.rounds(X.astype(np.float64), "average"), _rtol(prec))
    st = got["stats"]
    assert st["dense_k"] == n and st["dense_rounds"] == st["rounds"]
    assert st["dense_point_pairs"] == n * (n - 1) // 2


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("switch", [64, 700, 3000])
def test_dense_switch_in_mid_run(switch, prec, monkeypatch):
    """The range-query search (with the cache) first, then the matrix from the
    first round with at most `switch` active clusters; the sweep then visits
    exactly the point pairs in different clusters of that round."""
    monkeypatch.setenv("HAC_DENSE_K", str(switch))
    X = inputs.workload("gmm5d_1m_f32", n=6000)
    got = hac.cluster(X, "average", precision=prec, cache_slots=16)
    want = oracle.rounds(X.astype(np.float64), "average")
    _same(got, want, _rtol(prec))
    st = got["stats"]
    assert 0 < st["dense_k"] <= switch and 0 < st["dense_rounds"] < st["rounds"]
    # cluster sizes at the start of the first dense round, from the oracle's rounds
    r0 = st["rounds"] - st["dense_rounds"]
    sizes = {i: 1 for i in range(len(X))}
    for t in np.argsort(want["round"], kind="stable"):
        if want["round"][t] >= r0:
            break
        a, b = int(want["a"][t]), int(want["b"][t])
        sizes[a] += sizes.pop(b)
    assert len(sizes) == st["dense_k"]
    sz = np.array(list(sizes.values()), dtype=np.int64)
    assert st["dense_point_pairs"] == (sz.sum() ** 2 - (sz * sz).sum()) // 2


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_dense_exact_ties(prec, monkeypatch):
    """Lattice points (exact distance ties, duplicate points): a valid greedy
    tree with every merge within 1e-9 of the smallest active distance, and in
    the FP32 mode exactly the all-FP64 tree."""
    monkeypatch.setenv("HAC_DENSE_K", "65536")
    for seed, (n, dd, lev) in enumerate([(500, 3, 12), (800, 2, 6), (400, 4, 10)]):
        X = inputs.lattice(n, dd, seed=seed, levels=lev)
        got = hac.cluster(X, "average", precision=prec)
        bad, stats = oracle.validate(X.astype(np.float64), "average", got, rtol=1e-9,
                                     htol=_rtol(prec))
        assert bad == 0, stats
        if prec == hac.PREC_F32_RECHECK:
            ref = hac.cluster(X, "average", precision=hac.PREC_F64)
            _same(got, ref, 1e-5)
            assert got["stats"]["dense_rechecks"] > 0


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_dense_deterministic(prec, monkeypatch):
    """Sums are accumulated in fixed point by integer atomics: bit-identical
    heights run after run, whatever order the tiles finish in."""
    monkeypatch.setenv("HAC_DENSE_K", "4000")
    X = inputs.gaussian_mixture(9000, 3, 12, seed=44)
    a = hac.cluster(X, "average", precision=prec)
    b = hac.cluster(X, "average", precision=prec)
    for k in ("a", "b", "size", "round"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["h"].view(np.int64), b["h"].view(np.int64))
    assert a["stats"]["dense_k"] > 0


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("shape", [(4000, 16), (3000, 10), (2500, 8)], ids=lambda s: f"n{s[0]}d{s[1]}")
def test_candidate_lists_match(shape, prec, monkeypatch):
    """Average linkage with the exhaustive candidate scan in place of the tree
    (the default for d > 8, forced here for d = 8 too) and no dense matrix:
    the oracle's tree, round for round; every search scanned every cluster
    (a terminal whose list overflows searches the tree as well)."""
    monkeypatch.setenv("HAC_DENSE_K", "0")
    monkeypatch.setenv("HAC_BRUTE", "1")
    n, d = shape
    X = inputs.gaussian_mixture(n, d, 7, seed=n + d)
    got = hac.cluster(X, "average", precision=prec, cache_slots=32)
    _same(got, oracle.rounds(X.astype(np.float64), "average"), _rtol(prec))
    st = got["stats"]
    assert st["leaf_tests"] >= st["naive_pairs"]
