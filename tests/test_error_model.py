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


def _dense_estimate(A, B, k, es, sign):
    """The dense sweep's FP32 estimate of the mean distance of two clusters of
    float32 points: coordinates times 2^k, every FP32 step rounded, squared
    distances below 2^-126 flushed to zero before the approximate root,
    partial sums of at most 32 roots, each truncated to the unit 2^es."""
    s = F(2.0 ** k)
    As, Bs = (A * s).astype(F), (B * s).astype(F)
    total = 0
    for a in As:
        acc = np.zeros(len(Bs), F)
        for kk in range(A.shape[1]):
            t = (a[kk] - Bs[:, kk]).astype(F)
            acc = (acc + (t * t).astype(F)).astype(F)
        acc[acc < F(2.0 ** -126)] = 0
        roots = (np.sqrt(acc.astype(np.float64)) * (1.0 + sign * 2.0 ** -23)).astype(F)
        for g in range(0, len(roots), 32):
            part = F(0)
            for v in roots[g:g + 32]:
                part = F(part + v)
            total += int(np.floor(float(part) / 2.0 ** es))
    return total * 2.0 ** (es - k) / (len(A) * len(B))


def _dense_fp64(A, B, e):
    """The FP64 entry: every FP64 point distance truncated to the unit 2^e."""
    d = np.sqrt(((A[:, None, :].astype(np.float64) - B[None, :, :]) ** 2).sum(-1))
    return float(np.floor(d / 2.0 ** e).sum()) * 2.0 ** e / d.size


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1.0, 1e5, 1e11])
def test_dense_sweep_absolute_term(scale):
    """Dense-phase estimates against the FP64 entries they stand in for:
    |x - D| <= rho D + eta, rho = (d + 48) u, eta = 2 * 2^e + 2^(-63-k),
    with the sweep's scale 2^k (|coordinate| toward 2^40, 0 <= k <= 100) and
    unit e of a 10^6-point layout; clusters at every scale below the FP32
    paths' limit of 2^40, including near-duplicate points whose squared
    distances underflow unscaled."""
    rng = np.random.default_rng(int(np.log10(scale)) + 400)
    d, n = 5, 10 ** 6
    for trial in range(6):
        na, nb = rng.integers(1, 70, size=2)
        ca = rng.normal(size=d) * scale
        A = (ca + rng.normal(size=(na, d)) * scale * 10.0 ** -rng.integers(0, 9)).astype(F)
        B = (ca + rng.normal(size=d) * scale * 10.0 ** -rng.integers(0, 9)
             + rng.normal(size=(nb, d)) * scale * 10.0 ** -rng.integers(0, 9)).astype(F)
        pmax = float(max(np.abs(A).max(), np.abs(B).max()))
        k = max(0, min(100, 40 - int(np.ceil(np.log2(pmax))))) if pmax > 0 else 0
        dmax = 2.0 * pmax * np.sqrt(d) * (1 + 1e-5)
        e = int(np.floor(np.log2(0.25 * n * n * dmax))) + 1 - 126
        D = _dense_fp64(A, B, e)
        eta = (2.0 * 2.0 ** e + 2.0 ** (-63 - k)) * (1 + 1e-9)
        rho = (d + 48) * U
        for sign in (1.0, -1.0):
            x = _dense_estimate(A, B, k, e + k, sign)
            assert abs(x - D) <= rho * D + eta, (scale, trial, x, D, eta)


def test_dense_sweep_flush_near_origin():
    """Clusters of points within 1e-32 of the origin in a layout whose largest
    coordinate is 1 (so the sweep's scale is 2^40): their scaled squared
    distances fall below 2^-126 and flush to zero; the estimate stays within
    the absolute term 2^(-63-k)."""
    d, n = 3, 10 ** 6
    A = np.array([[0, 0, 0], [1e-32, 0, 0], [0, 3e-33, 0]], F)
    B = np.array([[2e-32, 1e-32, 0], [5e-33, 5e-33, 5e-33]], F)
    pmax, k = 1.0, 40
    dmax = 2.0 * pmax * np.sqrt(d) * (1 + 1e-5)
    e = int(np.floor(np.log2(0.25 * n * n * dmax))) + 1 - 126
    D = _dense_fp64(A, B, e)
    eta = (2.0 * 2.0 ** e + 2.0 ** (-63 - k)) * (1 + 1e-9)
    s = F(2.0 ** k)
    assert ((A[0] * s - B[1] * s).astype(F) ** 2).sum() < 2.0 ** -126  # the flush occurs
    for sign in (1.0, -1.0):
        x = _dense_estimate(A, B, k, e + k, sign)
        assert abs(x - D) <= (d + 48) * U * D + eta
