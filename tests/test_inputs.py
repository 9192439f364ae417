"""Seeded input generators: determinism and the stated shapes of each recipe."""
import math

import numpy as np
import pytest

from paper_2106_04727_gb300 import inputs


def test_counter_streams_are_deterministic_and_independent():
    a = inputs.uniform(7, 1, 1000)
    assert np.array_equal(a, inputs.uniform(7, 1, 1000))
    assert not np.array_equal(a, inputs.uniform(7, 2, 1000))
    assert not np.array_equal(a, inputs.uniform(8, 1, 1000))
    assert a.min() >= 0.0 and a.max() < 1.0
    z = inputs.normal(3, 4, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_uniform_fill_shape():
    n, d = 40000, 2
    X = inputs.uniform_fill(n, d, seed=1)
    side = math.sqrt(n)
    assert X.shape == (n, d) and X.dtype == np.float32
    assert X.min() >= 0.0 and X.max() <= side
    # uniform: each half of the box holds about half the points
    assert abs((X[:, 0] < side / 2).mean() - 0.5) < 0.01


def test_gaussian_disc_shape():
    n, d = 50000, 2
    X = inputs.gaussian_disc(n, d, seed=2).astype(np.float64)
    side = 5 * math.sqrt(n)
    assert X.shape == (n, d)
    assert X.min() >= 0.0 and X.max() <= side
    # five dense discs of standard deviation sqrt(n)/6 hold 90% of the points:
    # most points have a neighbour far closer than in a uniform fill
    g = np.floor(X / (math.sqrt(n) / 6)).astype(np.int64)
    cells, counts = np.unique(g[:, 0] * 100000 + g[:, 1], return_counts=True)
    assert np.sort(counts)[::-1][:5].sum() > 0.1 * n
    assert len(inputs.workload("gaussiandisc2d_1m_f32", n=1000)) == 1000


@pytest.mark.parametrize("name", sorted(inputs.WORKLOADS))
def test_named_workloads_small(name):
    X = inputs.workload(name, n=500)
    assert X.shape[0] == 500 and np.all(np.isfinite(X))
    assert np.array_equal(X, inputs.workload(name, n=500))
