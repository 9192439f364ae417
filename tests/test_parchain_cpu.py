"""The multithreaded CPU NN-chain (oracle/hac_parchain_cpu.c), the CPU
baseline at sizes the matrix oracle cannot hold, pinned to the matrix
oracle: Algorithm 1's rounds merge for merge (same pairs, sizes and round,
heights within 1e-12) on random inputs for every linkage, a valid greedy tree
on exact-tie lattices, the same result for any thread count, and a clean stop
between rounds at its time limit."""
import numpy as np
import pytest

import oracle
from paper_2106_04727_gb300 import inputs

LKS = ["complete", "average", "ward", "average_sq"]


def _rounds(d):
    out = {}
    for a, b, r in zip(d["a"], d["b"], d["round"]):
        out.setdefault(int(r), set()).add((int(a), int(b)))
    return out


@pytest.mark.parametrize("lk", LKS)
@pytest.mark.parametrize("shape", [(2, 1), (3, 2), (257, 2), (1500, 3), (900, 5), (400, 16)],
                         ids=lambda s: f"n{s[0]}d{s[1]}")
def test_same_rounds_as_oracle(lk, shape):
    n, d = shape
    X = inputs.gaussian_mixture(n, d, 6, seed=n + 7 * d).astype(np.float64)
    got = oracle.parchain_cpu(X, lk, threads=3)
    want = oracle.rounds(X, lk)
    assert got["complete"]
    c = oracle.compare(got, want, rtol=1e-12)
    assert c["ok"], c
    assert _rounds(got) == _rounds(want) and got["n_rounds"] == want["n_rounds"]


@pytest.mark.parametrize("lk", LKS)
def test_workload_sample(lk):
    """The benchmark's 10^6-point recipe at 5,000 points."""
    X = inputs.workload("gmm5d_1m_f32", n=5000).astype(np.float64)
    got = oracle.parchain_cpu(X, lk)
    c = oracle.compare(got, oracle.rounds(X, lk), rtol=1e-12)
    assert c["ok"], c


@pytest.mark.parametrize("lk", ["average", "ward", "average_sq", "complete"])
def test_exact_ties_valid(lk):
    X = inputs.lattice(400, 3, seed=11, levels=8).astype(np.float64)
    got = oracle.parchain_cpu(X, lk)
    bad, stats = oracle.validate(X, lk, got, rtol=1e-9)
    assert bad == 0, stats


def test_thread_count_does_not_change_the_result():
    X = inputs.gaussian_mixture(3000, 4, 9, seed=5).astype(np.float64)
    for lk in LKS:
        a = oracle.parchain_cpu(X, lk, threads=1)
        b = oracle.parchain_cpu(X, lk, threads=8)
        for k in ("a", "b", "size", "round"):
            assert np.array_equal(a[k], b[k]), (lk, k)
        assert np.array_equal(a["h"].view(np.int64), b["h"].view(np.int64))


def test_time_limit_stops_between_rounds():
    X = inputs.gaussian_mixture(20000, 5, 16, seed=2).astype(np.float64)
    got = oracle.parchain_cpu(X, "average", timeout_s=1e-9)
    assert not got["complete"] and got["n_rounds"] <= 1
    full = oracle.parchain_cpu(X[:300], "average", timeout_s=0.0)
    assert full["complete"] and len(full["a"]) == 299
