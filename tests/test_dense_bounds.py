"""The dense phase's bounds on an FP32-mode estimate, checked on the CPU.

An entry x of the matrix estimates the FP64 value D with
|x - D| <= delta + rho D + eta (csrc/hac_dense.cu, NNArgs).  The row scans
turn that into bounds in two ways, restated here from the host code of
dense_search and the scan kernel, and checked on random estimates that
satisfy the model with every error at its extreme:

  * FP64 arithmetic (delta > 0): lo = max(x - dl (1 + 2^-50), 0)
    (1 - 1e-12) / (1 + rho), up = (x + dl) (1 + 1e-12) / (1 - rho),
    dl = delta + eta (the 2^-50 covers the rounding of x - dl when x is
    close to dl, which the relative 1e-12 does not);
  * integer steps of the FP64 bit pattern (delta = 0): for x >= m0 = 2^30 eta,
    lo = x - nl ulps and up = x + nu ulps with rho widened by 2^-30 (which
    covers eta there); below m0 the estimate spans [0, 2 m0].

Both must contain D; a dropped term (eta, the 2^-30 widening, the 2^-50)
makes some case fail."""
import math
import struct

import numpy as np
import pytest

U = 2.0 ** -24


def _bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def _val(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _params(d, e, k):
    rho = (d + 48.0) * 5.9604644775390625e-8
    eta = (2.0 * 2.0 ** e + 2.0 ** (-63 - k)) * (1.0 + 1e-9)
    rho_i = rho + 2.0 ** -30
    nu = math.ceil(math.ldexp(rho_i / (1.0 - rho_i), 53) * (1.0 + 1e-6)) + 2
    nl = 2 * (math.ceil(math.ldexp(rho_i, 53) * (1.0 + 1e-6)) + 2)
    m0 = math.ldexp(eta, 30)
    return rho, eta, nu, nl, _bits(m0), _bits(2.0 * m0)


def _cases(rng, rho, eta, m):
    # D over many magnitudes, from far below eta to far above it
    D = 10.0 ** rng.uniform(math.log10(eta) - 3, math.log10(eta) + 40, size=m)
    D[: m // 10] = 0.0
    eps = rng.choice([-1.0, 1.0], size=m) * rng.uniform(0.9, 1.0, size=m) * rho
    abs_err = rng.choice([-1.0, 1.0], size=m) * rng.uniform(0.0, 1.0, size=m) * eta
    x = np.maximum(D * (1.0 + eps) + abs_err, 0.0)
    return D, x


@pytest.mark.parametrize("d,e,k", [(2, -80, 40), (5, -87, 38), (16, -60, 0), (5, -1000, 100)])
def test_integer_bounds_contain_the_fp64_value(d, e, k):
    rho, eta, nu, nl, m0, m0up = _params(d, e, k)
    assert rho + 2.0 ** -30 <= 4e-6  # the integer mode's condition on the host
    rng = np.random.default_rng(d * 1000 - e)
    D, x = _cases(rng, rho, eta, 20000)
    for Di, xi in zip(D, x):
        m = _bits(float(xi))
        lo = 0 if m < m0 else m - nl
        up = m0up if m < m0 else m + nu
        assert _val(lo) <= Di <= _val(up), (Di, xi)


@pytest.mark.parametrize("d,delta", [(2, 1e-3), (5, 0.0), (16, 7.5)])
def test_fp64_bounds_contain_the_fp64_value(d, delta):
    rho, eta, _, _, _, _ = _params(d, -70, 20)
    dl = delta + eta
    lo_f = (1.0 - 1e-12) / (1.0 + rho)
    up_f = (1.0 + 1e-12) / (1.0 - rho)
    rng = np.random.default_rng(int(d + 10 * delta))
    D = 10.0 ** rng.uniform(-30, 10, size=20000)
    eps = rng.choice([-1.0, 1.0], size=D.size) * rho
    a = rng.choice([-1.0, 1.0], size=D.size) * dl
    x = np.maximum(D * (1.0 + eps) + a, 0.0)
    lo = np.maximum(x - dl * (1.0 + 2.0 ** -50), 0.0) * lo_f
    up = (x + dl) * up_f
    assert np.all(lo <= D) and np.all(D <= up)


def test_fp64_lower_bound_needs_the_absolute_widening():
    """Without the 2^-50 widening, an estimate just above dl (D far below
    dl) gives a lower bound above D: the rounding of x - dl is absolute."""
    rho, eta, _, _, _, _ = _params(5, -70, 20)
    lo_f = (1.0 - 1e-12) / (1.0 + rho)
    D = 3.703202768806104e-28
    x = D * (1.0 + rho) + eta
    assert max(x - eta, 0.0) * lo_f > D
    assert max(x - eta * (1.0 + 2.0 ** -50), 0.0) * lo_f <= D


def test_a_missing_term_is_caught():
    """Planted mistakes, each caught at the model's extreme: integer bounds
    without the absolute term (every estimate on relative steps), and steps
    from rho alone (no 2^-30 widening) at the top of a binade just above
    m0, where eta is 2^-30 of the entry."""
    d, e, k = 5, -87, 38
    rho, eta, nu, nl, m0, m0up = _params(d, e, k)
    # (1) relative steps only: an estimate of 2 eta for D = 3 eta
    D = 3.0 * eta
    x = D * (1.0 - rho) - eta
    m = _bits(x)
    assert _val(m + nu) < D                 # the mistake misses D ...
    assert m < m0 and _val(m0up) >= D       # ... the kept rule spans it
    # (2) nu from rho alone
    nu0 = math.ceil(math.ldexp(rho / (1.0 - rho), 53) * (1.0 + 1e-6)) + 2
    # nu0 ulps below a power of two: the steps up stay in the smaller-ulp
    # binade, the least relative increase
    top = _bits(2.0 ** math.ceil(math.log2(_val(m0)) + 1)) - nu0
    x = _val(top)
    assert top >= m0
    eta_x = x * 2.0 ** -30                  # the largest eta with x >= m0 = 2^30 eta
    D = (x + eta_x) / (1.0 - rho)
    assert _val(top + nu0) < D
    rho_i = rho + 2.0 ** -30
    nu_i = math.ceil(math.ldexp(rho_i / (1.0 - rho_i), 53) * (1.0 + 1e-6)) + 2
    assert _val(top + nu_i) >= D
