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
