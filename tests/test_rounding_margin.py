"""The rounding margin of the float lower bound, checked on the CPU.

The float kernels evaluate a clamp distance as in ``box_dist_f32``
(``kc_device.cuh``): per attribute one correctly rounded subtraction of each
side, ``(lo - x, x - hi)``, the larger of the two and 0, then the squares
accumulated by fused multiply-adds in two interleaved chains (even attributes
in one, odd in the other; an odd last attribute joins the first), and one
final add.  The proved bound is ``|d' - d| <= gamma_n d`` with
``n = ceil(D/2) + 3`` and ``gamma_n = n u / (1 - n u)``, ``u = 2^-24``; the
certified value ``RD(RD(d' (1 - gamma_n)(1 - 2^-51)) - (D + 2) 2^-149)`` is
then never above ``d`` and at most ``2 gamma_n`` below it.

Here that evaluation order is emulated with correctly rounded float32
operations (fused multiply-adds rounded once, from an exact two-sum) and the
certified value is compared with ``d`` in exact rational arithmetic, on
random inputs spread over six decades (so that subtractions round) and on
inputs built so that every subtraction rounds up.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -24


def gamma(n):
    return n * U / (1 - n * U)


def roundings(d):
    return 2 + (d + 1) // 2 + 1


def fma32(a, b, c):
    """float32 a*b + c rounded once (a, b, c float32 arrays, normal range)."""
    p = a.astype(np.float64) * b.astype(np.float64)          # exact: 24 + 24 bits
    q = c.astype(np.float64)
    s = p + q
    bb = s - p
    e = (p - (s - bb)) + (q - bb)                             # s + e == p + q exactly
    r = s.astype(np.float32)
    # s may sit exactly halfway between two floats while s + e does not
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    lo_n = np.where(r.astype(np.float64) > s, dn, r)
    hi_n = np.where(r.astype(np.float64) > s, r, up)
    tie = (s - lo_n.astype(np.float64)) == (hi_n.astype(np.float64) - s)
    fix = tie & (e != 0)
    r = np.where(fix & (e > 0), hi_n, np.where(fix & (e < 0), lo_n, r))
    return r.astype(np.float32)


def box_dist_f32(x, lo, hi):
    """The kernels' float clamp distance for rows of x, lo, hi (T, D)."""
    T, D = x.shape
    acc0 = np.zeros(T, np.float32)
    acc1 = np.zeros(T, np.float32)
    m = np.maximum(np.maximum(lo - x, x - hi), np.float32(0))   # float32 subtractions
    for a in range(0, D - 1, 2):
        acc0 = fma32(m[:, a], m[:, a], acc0)
        acc1 = fma32(m[:, a + 1], m[:, a + 1], acc1)
    if D % 2:
        acc0 = fma32(m[:, D - 1], m[:, D - 1], acc0)
    return (acc0 + acc1).astype(np.float32)


def round_down(q):
    f = float(q)
    if Fraction(f) > q:
        f = math.nextafter(f, -math.inf)
    return f


def certified(dprime, D):
    g = gamma(roundings(D))
    defl = (1.0 - g) * (1.0 - 4 * 2.0 ** -53)
    v = round_down(Fraction(float(dprime)) * Fraction(defl))
    return round_down(Fraction(v) - Fraction(D + 2) * Fraction(2.0 ** -149))


def exact(x, lo, hi):
    s = Fraction(0)
    for xa, la, ha in zip(x.tolist(), lo.tolist(), hi.tolist()):
        fx, fl, fh = Fraction(xa), Fraction(la), Fraction(ha)
        t = max(fl - fx, fx - fh, Fraction(0))
        s += t * t
    return s


def _check(x, lo, hi):
    D = x.shape[1]
    g = gamma(roundings(D))
    dp = box_dist_f32(x, lo, hi)
    worst = 0.0
    for i in range(x.shape[0]):
        d = exact(x[i], lo[i], hi[i])
        c = certified(dp[i], D)
        assert Fraction(c) <= d, (D, i)
        if d > 0:
            rel = float((Fraction(float(dp[i])) - d) / d)
            worst = max(worst, abs(rel))
            assert abs(rel) <= g
            assert float((d - Fraction(c)) / d) <= 2 * g + 1e-15
    return worst


def _round32(q):
    """Nearest float32 to a positive Fraction, ties to even."""
    f = np.float32(float(q))
    cands = [np.nextafter(f, np.float32(0)), f, np.nextafter(f, np.float32(np.inf))]
    return min(cands, key=lambda v: (abs(Fraction(float(v)) - q), int(np.float32(v).view(np.uint32)) & 1))


def test_fused_multiply_add_emulation_is_rounded_once():
    rng = np.random.default_rng(0)
    a = (10.0 ** rng.uniform(-3, 3, 4000)).astype(np.float32)
    c = (10.0 ** rng.uniform(-6, 6, 4000)).astype(np.float32)
    r = fma32(a, a, c)
    for i in range(len(a)):
        assert r[i] == _round32(Fraction(float(a[i])) ** 2 + Fraction(float(c[i])))


def _spread(rng, shape):
    return (rng.choice([-1.0, 1.0], size=shape) * 10.0 ** rng.uniform(-3, 3, size=shape)).astype(np.float32)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 8, 13, 16])
def test_margin_on_spread_inputs(D):
    rng = np.random.default_rng(D)
    T = 1500
    x = _spread(rng, (T, D))
    lo = _spread(rng, (T, D))
    hi = (lo.astype(np.float64) + np.abs(_spread(rng, (T, D)))).astype(np.float32)
    hi = np.maximum(hi, lo)
    inside = rng.uniform(size=(T, D)) < 0.2        # some attributes inside the box
    lo = np.where(inside, np.minimum(lo, x), lo)
    hi = np.where(inside, np.maximum(hi, x), hi)
    worst = _check(x, lo, hi)
    # the inputs do exercise the roundings: the worst error seen is 2.8-4.0 u
    # (4.0 u at D = 4 against the bound gamma_5 = 5 u)
    assert worst > 2 * U


@pytest.mark.parametrize("D", [2, 8, 16])
def test_margin_when_every_subtraction_rounds_up(D):
    """Boxes far above x, and x nudged down one float at a time until the
    float difference lo - x rounds up: (nearly) every rounded difference
    exceeds the real one, the direction the deflation has to absorb."""
    rng = np.random.default_rng(100 + D)
    T = 800
    x = rng.uniform(1e-3, 2e-3, size=(T, D)).astype(np.float32)
    big = rng.uniform(1.0, 2.0, size=(T, D)).astype(np.float32)
    # keep pairs whose float difference rounds up
    diff = (big - x).astype(np.float64)
    exact_diff = big.astype(np.float64) - x.astype(np.float64)
    for _ in range(50):
        bad = diff < exact_diff
        if not bad.any():
            break
        x = np.where(bad, np.nextafter(x, np.float32(0)), x)
        diff = (big - x).astype(np.float64)
        exact_diff = big.astype(np.float64) - x.astype(np.float64)
    assert np.mean(diff > exact_diff) > 0.5
    lo = big
    hi = (big + np.float32(1.0)).astype(np.float32)
    _check(x, lo, hi)
