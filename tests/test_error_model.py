"""The FP32 error model of the search and pair kernels, checked on the CPU
by emulating their float32 arithmetic with numpy (every subtract, multiply
and add rounded separately, which is never better than the kernels' fused
multiply-adds) against FP64 on random and adversarial inputs:

    |D32 - D| <= delta + rho * D,   rho = (d + 16) u  (+ 32 u for average),
    delta = 0 for point distances of float32 input, 2.01 u M sqrt(d) when
    float64 coordinates (|x| <= M after recentring) are rounded to float32,
    times sqrt(2|A||B|/(|A|+|B|)) for Ward's centroid form; u = 2^-24.

Square roots are also perturbed by a relative 2^-23 in either direction,
beyond the rounding of a correctly rounded root, as a margin for the
approximate root the GPU-wide kernels take."""
import numpy as np
import pytest

U = 2.0 ** -24
F = np.float32


def _d32_rows(X32, Y32, sqrt_err=0.0, sign=1.0):
    """FP32 distances of row pairs: rounded differences, squares and sums."""
    acc = np.zeros(len(X32), F)
    for k in range(X32.shape[1]):
        t = (X32[:, k] - Y32[:, k]).astype(F)
        acc = (acc + (t * t).astype(F)).astype(F)
    r = np.sqrt(acc).astype(np.float64)
    return r * (1.0 + sign * sqrt_err)


def _exact(X, Y):
    return np.sqrt(((X.astype(np.float64) - Y.astype(np.float64)) ** 2).sum(1))


def _cases(rng, d, m):
    scale = 10.0 ** rng.uniform(-3, 6, size=(m, 1))
    X = rng.normal(size=(m, d)) * scale
    # half the pairs nearly coincide (cancellation), the rest are far apart
    close = rng.random(m) < 0.5
    Y = np.where(close[:, None], X + rng.normal(size=(m, d)) * scale * 1e-5,
                 rng.normal(size=(m, d)) * scale)
    return X, Y


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 10, 16])
def test_float32_input_points(d):
    rng = np.random.default_rng(d)
    X, Y = _cases(rng, d, 40000)
    X32, Y32 = X.astype(F), Y.astype(F)
    D = _exact(X32, Y32)  # the input IS the float32 data: delta = 0
    rho = (d + 16) * U
    for sign in (1.0, -1.0):
        D32 = _d32_rows(X32, Y32, sqrt_err=2.0 ** -23, sign=sign)
        assert np.all(np.abs(D32 - D) <= rho * D + 1e-300)


@pytest.mark.parametrize("d", [1, 2, 5, 16])
def test_float64_input_rounded_to_float32(d):
    rng = np.random.default_rng(100 + d)
    X, Y = _cases(rng, d, 40000)
    ctr = 0.5 * (np.minimum(X.min(0), Y.min(0)) + np.maximum(X.max(0), Y.max(0)))
    Xc, Yc = X - ctr, Y - ctr  # recentred in FP64, then rounded
    M = max(np.abs(Xc).max(), np.abs(Yc).max())
    D = _exact(Xc, Yc)
    D32 = _d32_rows(Xc.astype(F), Yc.astype(F), sqrt_err=2.0 ** -23)
    delta = 2.01 * U * M * np.sqrt(d)
    assert np.all(np.abs(D32 - D) <= delta + (d + 16) * U * D)


@pytest.mark.parametrize("d", [2, 5])
def test_average_partial_sums(d):
    """Mean of point distances: float32 partial sums of at most 32 terms,
    each added to an FP64 accumulator."""
    rng = np.random.default_rng(200 + d)
    for _ in range(30):
        na, nb = rng.integers(1, 90, size=2)
        A = (rng.normal(size=(na, d)) * 50).astype(F)
        B = (rng.normal(size=(nb, d)) * 50 + rng.normal(size=d) * 20).astype(F)
        ii, jj = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
        terms = _d32_rows(A[ii.ravel()], B[jj.ravel()], sqrt_err=2.0 ** -23).astype(F)
        acc = 0.0
        for g in range(0, len(terms), 32):
            part = F(0)
            for v in terms[g:g + 32]:
                part = F(part + v)
            acc += float(part)
        D32 = acc / (na * nb)
        D = _exact(A[ii.ravel()], B[jj.ravel()]).mean()
        assert abs(D32 - D) <= (d + 16 + 32) * U * D


@pytest.mark.parametrize("d", [2, 5, 16])
def test_ward_centroid_form(d):
    """Ward from float32-rounded FP64 centroids: D32 = sqrt(w * dc2) with the
    weight w = 2|A||B| / (|A|+|B|) formed in FP32 (rounded product, rounded
    reciprocal, rounded product) and dc2 the FP32 squared centroid gap; delta
    scales with sqrt(w)."""
    rng = np.random.default_rng(300 + d)
    m = 20000
    ca = rng.normal(size=(m, d)) * 10.0 ** rng.uniform(-2, 5, size=(m, 1))
    cb = ca + rng.normal(size=(m, d)) * 10.0 ** rng.uniform(-6, 5, size=(m, 1))
    na = rng.integers(1, 10 ** 6, size=m).astype(np.float64)
    nb = rng.integers(1, 10 ** 6, size=m).astype(np.float64)
    M = max(np.abs(ca).max(), np.abs(cb).max())
    w = 2 * na * nb / (na + nb)
    D = np.sqrt(w) * _exact(ca, cb)
    na32, nb32 = na.astype(F), nb.astype(F)
    rcp = (1.0 / (na32 + nb32).astype(F).astype(np.float64)).astype(F)
    w32 = ((F(2) * na32 * nb32).astype(F) * rcp).astype(F)
    X32, Y32 = ca.astype(F), cb.astype(F)
    dc2 = np.zeros(m, F)
    for k in range(d):
        t = (X32[:, k] - Y32[:, k]).astype(F)
        dc2 = (dc2 + (t * t).astype(F)).astype(F)
    D32 = np.sqrt((w32 * dc2).astype(F)).astype(np.float64)
    delta = 2.01 * U * M * np.sqrt(d) * np.sqrt(w)
    assert np.all(np.abs(D32 - D) <= delta + (d + 16) * U * D)
