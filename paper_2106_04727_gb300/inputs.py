"""Seeded synthetic point sets for the HAC workloads.

This module holds random-number generation and workload shapes only: no
distance, linkage or clustering arithmetic.  Both the CPU oracle tests and the
GPU path draw their inputs from here, so the two sides see identical points.

Randomness is a counter-based SplitMix64 stream (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): output ``i`` of
stream ``(seed, stream)`` is the SplitMix64 finaliser applied to
``key + (i + 1) * 0x9E3779B97F4A7C15`` where ``key`` mixes the seed and stream
id.  It is pure uint64 arithmetic, so the same seed gives the same points on
x86 and on Arm, independent of numpy's own generators.

Workloads follow the shapes the ParChain paper evaluates (Section 6,
"Data Sets": low-dimensional, 10^6-10^7 points, Gaussian clusters plus
uniform noise); the paper's real data sets are not used.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
        b = _mix(np.array([(stream * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF],
                          dtype=np.uint64) ^ a)
    return b[0]


def u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit outputs of stream ``(seed, stream)`` from ``offset``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
        return _mix(_key(seed, stream) + i * _GOLDEN)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, 2 * stream + 1000003, count)
    u2 = uniform(seed, 2 * stream + 1000004, count)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def randint(seed: int, stream: int, count: int, high: int) -> np.ndarray:
    """Integers in [0, high) (floor of a uniform draw)."""
    return np.minimum((uniform(seed, stream, count) * high).astype(np.int64), high - 1)


# ----------------------------------------------------------------------------
# Workload shapes
# ----------------------------------------------------------------------------

def uniform_cube(n: int, d: int, seed: int, lo: float = 0.0, hi: float = 1.0,
                 dtype=np.float64) -> np.ndarray:
    """i.i.d. uniform points in [lo, hi)^d."""
    x = lo + (hi - lo) * uniform(seed, 1, n * d)
    return np.ascontiguousarray(x.reshape(n, d).astype(dtype))


def gaussian_mixture(n: int, d: int, k: int, seed: int, box: float = 100.0,
                     sigma_lo: float = 0.5, sigma_hi: float = 3.0,
                     dtype=np.float32) -> np.ndarray:
    """Mixture of ``k`` isotropic Gaussians with equal weights.

    Centres are uniform in [0, box]^d, each component's sigma is uniform in
    [sigma_lo, sigma_hi], and each point picks its component by one
    categorical draw.
    """
    centers = box * uniform(seed, 11, k * d).reshape(k, d)
    sig = sigma_lo + (sigma_hi - sigma_lo) * uniform(seed, 12, k)
    comp = randint(seed, 13, n, k)
    z = normal(seed, 14, n * d).reshape(n, d)
    x = centers[comp] + sig[comp, None] * z
    return np.ascontiguousarray(x.astype(dtype))


def spreaders(n: int, seed: int, n_spreaders: int = 200, box: float = 1e5,
              sigma_lo: float = 1.0, sigma_hi: float = 50.0,
              noise_frac: float = 0.01, dtype=np.float32) -> np.ndarray:
    """Varying-density 2-D data: random-walk seed spreaders plus uniform noise.

    Each spreader starts uniform in [0, box]^2 with its own sigma in
    [sigma_lo, sigma_hi].  It emits a point at its position plus N(0, sigma^2 I)
    jitter, then steps by N(0, sigma^2 I); the walk is reflected at the box
    edges (folding a free walk gives the reflected walk).  99% of the points
    are split equally across spreaders, 1% are uniform noise in the box.
    """
    d = 2
    n_noise = int(round(n * noise_frac))
    n_walk = n - n_noise
    per = np.full(n_spreaders, n_walk // n_spreaders, dtype=np.int64)
    per[: n_walk - per.sum()] += 1
    start = box * uniform(seed, 21, n_spreaders * d).reshape(n_spreaders, d)
    sig = sigma_lo + (sigma_hi - sigma_lo) * uniform(seed, 22, n_spreaders)
    owner = np.repeat(np.arange(n_spreaders), per)
    first = np.concatenate([[0], np.cumsum(per)[:-1]])
    steps = normal(seed, 23, n_walk * d).reshape(n_walk, d) * sig[owner, None]
    # position before emitting point j of spreader s: start + sum of earlier steps
    csum = np.cumsum(steps, axis=0)
    base = csum[first] - steps[first]          # cumulative sum just before each walk
    walk = start[owner] + (csum - steps) - base[owner]
    period = 2.0 * box
    walk = np.mod(walk, period)
    walk = np.where(walk > box, period - walk, walk)
    jitter = normal(seed, 24, n_walk * d).reshape(n_walk, d) * sig[owner, None]
    pts = np.empty((n, d), dtype=np.float64)
    pts[:n_walk] = walk + jitter
    pts[n_walk:] = box * uniform(seed, 25, n_noise * d).reshape(n_noise, d)
    perm = np.argsort(u64(seed, 26, n), kind="stable")   # interleave noise and walks
    return np.ascontiguousarray(pts[perm].astype(dtype))


def lattice(n: int, d: int, seed: int, levels: int = 1024, step: float = 1.0 / 256,
            dtype=np.float32) -> np.ndarray:
    """Coordinates floor(U[0,1) * levels) * step: a 2^-8 lattice in [0, 4)^d.

    Every coordinate and every squared difference is exactly representable
    in FP32, so equal point distances are equal in any precision.
    """
    k = randint(seed, 31, n * d, levels).astype(np.float64)
    return np.ascontiguousarray((k * step).reshape(n, d).astype(dtype))


def uniform_fill(n: int, d: int, seed: int, dtype=np.float32) -> np.ndarray:
    """The paper's UniformFill shape (Section 6, data sets): n points uniform
    in a hypergrid of side sqrt(n)."""
    side = math.sqrt(n)
    return np.ascontiguousarray((side * uniform(seed, 61, n * d)).reshape(n, d).astype(dtype))


def gaussian_disc(n: int, d: int, seed: int, clusters: int = 5, frac: float = 0.9,
                  dtype=np.float32) -> np.ndarray:
    """The paper's GaussianDisc shape (Section 6, data sets): a hypergrid of
    side 5 sqrt(n); 90% of the points split equally among five Gaussian
    clusters with means uniform in the hypergrid and diameter sqrt(n) (read
    as standard deviation sqrt(n) / 6 per axis, clipped to the hypergrid);
    the other 10% uniform in the hypergrid.  Points are interleaved."""
    side = 5.0 * math.sqrt(n)
    sigma = math.sqrt(n) / 6.0
    m = int(round(frac * n))
    centers = side * uniform(seed, 62, clusters * d).reshape(clusters, d)
    comp = np.arange(m) % clusters
    pts = np.empty((n, d), dtype=np.float64)
    pts[:m] = np.clip(centers[comp] + sigma * normal(seed, 63, m * d).reshape(m, d), 0.0, side)
    pts[m:] = side * uniform(seed, 64, (n - m) * d).reshape(n - m, d)
    perm = np.argsort(u64(seed, 65, n), kind="stable")
    return np.ascontiguousarray(pts[perm].astype(dtype))


# ----------------------------------------------------------------------------
# Named workloads (sizes as the HAC benchmarks use them)
# ----------------------------------------------------------------------------

WORKLOADS = {
    # 1,024 uniform FP64 points in the unit square; all three linkages.
    "uniform2d_1k_f64": dict(kind="uniform", n=1024, d=2, seed=1000, dtype=np.float64),
    # 10^6 FP32 points, 64-component Gaussian mixture in [0,100]^5.
    "gmm5d_1m_f32": dict(kind="gmm", n=1_000_000, d=5, k=64, seed=2000, dtype=np.float32),
    # 10^7 FP32 points from 200 random-walk spreaders plus 1% noise in [0,1e5]^2.
    "spread2d_10m_f32": dict(kind="spreaders", n=10_000_000, seed=3000, dtype=np.float32),
    # 10^6 FP32 points on the 2^-8 lattice in [0,4)^16.
    "lattice16d_1m_f32": dict(kind="lattice", n=1_000_000, d=16, seed=5000, dtype=np.float32),
    # the paper's synthetic shapes (2U/2G/5U/5G at 10^6 and 10^7 points)
    "uniformfill2d_1m_f32": dict(kind="uniformfill", n=1_000_000, d=2, seed=6000),
    "gaussiandisc2d_1m_f32": dict(kind="gaussiandisc", n=1_000_000, d=2, seed=6100),
    "uniformfill5d_1m_f32": dict(kind="uniformfill", n=1_000_000, d=5, seed=6200),
    "gaussiandisc5d_1m_f32": dict(kind="gaussiandisc", n=1_000_000, d=5, seed=6300),
    "uniformfill2d_10m_f32": dict(kind="uniformfill", n=10_000_000, d=2, seed=6400),
    "gaussiandisc2d_10m_f32": dict(kind="gaussiandisc", n=10_000_000, d=2, seed=6500),
    "uniformfill5d_10m_f32": dict(kind="uniformfill", n=10_000_000, d=5, seed=6600),
    "gaussiandisc5d_10m_f32": dict(kind="gaussiandisc", n=10_000_000, d=5, seed=6700),
}


def make(kind: str, n: int, d: int = 2, seed: int = 0, k: int = 64,
         dtype=np.float32) -> np.ndarray:
    """Build one point set of the given kind and size."""
    if kind == "uniform":
        return uniform_cube(n, d, seed, dtype=dtype)
    if kind == "gmm":
        return gaussian_mixture(n, d, k, seed, dtype=dtype)
    if kind == "spreaders":
        return spreaders(n, seed, dtype=dtype)
    if kind == "lattice":
        return lattice(n, d, seed, dtype=dtype)
    if kind == "uniformfill":
        return uniform_fill(n, d, seed, dtype=dtype)
    if kind == "gaussiandisc":
        return gaussian_disc(n, d, seed, dtype=dtype)
    raise ValueError(f"unknown workload kind {kind!r}")


def workload(name: str, n: int | None = None) -> np.ndarray:
    """A named workload, optionally truncated to its first ``n`` points' recipe.

    With ``n`` given, the same recipe is drawn at size ``n`` (a smaller sample
    of the same distribution, not a prefix of the full set).
    """
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    return make(**w)


def serving_requests(count: int, seed: int, n_lo: int = 64, n_hi: int = 65536,
                     dims=(2, 3, 5, 10)):
    """Parameters of a stream of independent HAC requests.

    n is log-uniform in [n_lo, n_hi], d uniform over ``dims``, linkage uniform
    over {complete, average, Ward} (0, 1, 2), and each request's points come
    from its own Gaussian mixture with 4-32 components.
    """
    u = uniform(seed, 41, count)
    ns = np.round(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)
    ds = np.asarray(dims)[randint(seed, 42, count, len(dims))]
    lks = randint(seed, 43, count, 3)
    ks = 4 + randint(seed, 44, count, 29)
    return [dict(n=int(ns[i]), d=int(ds[i]), linkage=int(lks[i]), k=int(ks[i]),
                 seed=seed * 100003 + i) for i in range(count)]


def request_points(req: dict) -> np.ndarray:
    """Points of one serving request (FP32 Gaussian mixture)."""
    return gaussian_mixture(req["n"], req["d"], req["k"], req["seed"], dtype=np.float32)
