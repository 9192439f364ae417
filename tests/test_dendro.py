"""The vectorised dendrogram checks used by the full-size GPU tests, on the CPU:
they accept every tree the oracle builds, reject the same planted mistakes as
the oracle's `check_tree`, and recover each merged cluster's points."""
import numpy as np
import pytest

import dendro
import oracle
from paper_2106_04727_gb300 import inputs


def _tree(lk, n=400, d=3, seed=4):
    X = inputs.gaussian_mixture(n, d, 6, seed=seed).astype(np.float64)
    return X, oracle.rounds(X, lk)


@pytest.mark.parametrize("lk", ["complete", "average", "ward", "average_sq"])
def test_accepts_oracle_trees(lk):
    X, t = _tree(lk)
    assert dendro.check(t, len(X)) == []
    assert oracle.check_tree(t, len(X)) == []


def test_degenerate_sizes():
    X = np.zeros((1, 2))
    assert dendro.check(oracle.rounds(X, "ward"), 1) == []
    X = np.array([[0.0, 0.0], [1.0, 0.0]])
    t = oracle.rounds(X, "average")
    assert dendro.check(t, 2) == []
    assert dendro.check(t, 3) != []


def _mutants(t):
    m = len(t["a"])
    big = int(np.argmax(t["size"]))
    ca, cb, _ = dendro.children(t)
    child = int(ca[big]) if ca[big] >= 0 else int(cb[big])
    out = {}
    c = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in t.items()}
    c["size"][big] -= 1
    out["size"] = c
    c = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in t.items()}
    c["h"][big] = c["h"][child] * 0.5
    out["height"] = c
    c = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in t.items()}
    c["a"], c["b"] = c["a"][:-1], c["b"][:-1]
    for k in ("h", "size", "round"):
        c[k] = c[k][:-1]
    out["count"] = c
    # a retired cid reused by a later merge
    c = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in t.items()}
    first = int(np.argmin(c["round"]))
    b0 = int(c["b"][first])
    late = int(np.flatnonzero((c["round"] > c["round"][first]) & (c["b"] > b0))[0])
    c["a"][late] = b0
    out["reuse"] = c
    assert m > 2
    return out


@pytest.mark.parametrize("kind", ["size", "height", "count", "reuse"])
def test_rejects_planted_mistakes(kind):
    X, t = _tree("average")
    bad = _mutants(t)[kind]
    assert dendro.check(bad, len(X)) != []
    assert oracle.check_tree(bad, len(X)) != []


def test_same_round_twice_rejected():
    X, t = _tree("complete")
    ca, _, _ = dendro.children(t)
    k = int(np.flatnonzero(ca >= 0)[0])
    c = {k2: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k2, v in t.items()}
    c["round"][k] = c["round"][ca[k]]
    assert dendro.check(c, len(X)) != []


@pytest.mark.parametrize("lk", ["complete", "average", "ward", "average_sq"])
def test_sampled_members_reproduce_heights(lk):
    """The point sets recovered for sampled merges give, through the Table 1
    definitions, the heights the Lance-Williams oracle recorded."""
    X, t = _tree(lk, n=600, seed=8)
    picks = dendro.sample_small(t, 40, cap=64, seed=1)
    assert len(picks) == 40
    for m, sa, sb in picks:
        assert len(sa) + len(sb) == t["size"][m]
        assert min(sa) == t["a"][m] and min(sb) == t["b"][m]
        want = oracle.cluster_dist(lk, X[sa], X[sb])
        assert t["h"][m] == pytest.approx(want, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("lk", ["complete", "average", "ward", "average_sq"])
def test_rnn_check_accepts_oracle_trees(lk):
    """Every merge of the oracle's Algorithm 1 joins reciprocal nearest
    neighbours among the clusters active in its round, and the partner
    distance from the points equals the recorded height."""
    X = inputs.gaussian_mixture(2500, 3, 8, seed=3).astype(np.float64)
    t = oracle.rounds(X, lk)
    picks = dendro.pick_merges(t, 40, cap=32, k_big=3, every_size=lk == "ward")
    probs, ties, vals = dendro.rnn_check(t, X, lk, picks, oracle.dist_to_all)
    assert probs == [] and len(vals) == len(picks)
    for m, v in vals.items():
        assert v == pytest.approx(t["h"][m], rel=1e-12)


def test_rnn_check_on_exact_ties():
    """Lattice points: exact ties among candidates are near ties, never
    problems, when the tree breaks them by the smaller cid."""
    X = inputs.lattice(500, 3, seed=2, levels=8).astype(np.float64)
    t = oracle.rounds(X, "ward")
    picks = dendro.pick_merges(t, 60, every_size=True)
    probs, ties, _ = dendro.rnn_check(t, X, "ward", picks, oracle.dist_to_all)
    assert probs == []


@pytest.mark.parametrize("lk", ["average", "ward"])
def test_rnn_check_catches_a_wrong_partner(lk):
    """A merge whose partner is replaced by a farther active cluster fails."""
    X = inputs.gaussian_mixture(1500, 2, 6, seed=9).astype(np.float64)
    t = oracle.rounds(X, lk)
    r0 = np.flatnonzero(t["round"] == 0)
    m = int(r0[0])
    # the active clusters of round 0 are the singletons: take a farther one
    q = int(t["a"][m])
    D = oracle.dist_to_all(lk, X, np.arange(len(X)), q)
    D[q] = np.inf
    far = int(np.argsort(D)[5])
    bad = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in t.items()}
    bad["b"][m] = far
    probs, _, _ = dendro.rnn_check(bad, X, lk, [m], oracle.dist_to_all)
    assert probs and "closer" in probs[0]


def test_sample_big_picks_the_most_pairs_within_the_limit():
    """Merges ((0,1), (2,3), (01,23), (0123,4)) of five points: pair counts
    1, 1, 4, 4; a limit of 3 leaves the first two; the largest within 4 are
    the last two, with their point sets."""
    d = {"a": np.array([0, 2, 0, 0]), "b": np.array([1, 3, 2, 4]),
         "h": np.array([1.0, 1.0, 2.0, 3.0]), "size": np.array([2, 2, 4, 5]),
         "round": np.array([0, 0, 1, 2])}
    got = dendro.sample_big(d, 2, 4)
    assert [t for t, _, _ in got] == [2, 3]
    assert sorted(got[0][1]) == [0, 1] and sorted(got[0][2]) == [2, 3]
    assert sorted(got[1][1]) == [0, 1, 2, 3] and got[1][2] == [4]
    assert [t for t, _, _ in dendro.sample_big(d, 2, 3)] == [0, 1]
