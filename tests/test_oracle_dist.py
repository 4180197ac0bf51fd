"""Pins of the oracle's non-uniform variates (exponential by inversion, normal
by Box & Muller 1958) from FP32 uniforms.  The paper covers uniform draws
only; these transforms are the first extension row.  The oracle writes ln,
sin and cos out from their series in single precision, so it is pinned here
against things it does not share: exact rationals for its constants, float64
libm over every one of the 2^24 FP32 uniforms a generator can return (error
bound derived below), exact values at the quadrant points, and distribution
tests of the variates."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

PI = Fraction("3.14159265358979323846264338327950288419716939937510582097494459")
LN2 = Fraction("0.69314718055994530941723212145817656807550013436025525412068000")
ALL_U = np.arange(1 << 24, dtype=np.float64) * 2.0**-24   # every FP32 uniform, exactly


def f32_round(x: Fraction) -> float:
    """x rounded to the nearest float32 (ties to even), decided in exact arithmetic."""
    c = np.float32(float(x))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - x)
        key = (d, int(np.array(cand).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return float(best[1])


def ulp_err(got, ref):
    """|got - ref| in units of the float32 spacing at |ref| (ref in float64)."""
    got = np.asarray(got, dtype=np.float64)
    sp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    return np.abs(got - ref) / sp


def test_constants_against_exact_rationals():
    k = O.dist_constants()
    hi = Fraction(math.floor(LN2 * 2**15), 2**15)
    assert Fraction(k["ln2_hi"]) == hi and hi.numerator.bit_length() <= 15
    assert k["ln2_lo"] == f32_round(LN2 - hi)
    for j in range(6):
        assert k["inv_odd"][j] == f32_round(Fraction(1, 2 * j + 1))
    half_pi = PI / 2
    for n in range(1, 11):
        exact = half_pi**n / math.factorial(n) * (-1 if (n // 2) % 2 else 1)
        assert k["sc"][n] == f32_round(exact), n


def test_exponential_exhaustive_within_two_ulp():
    """Every FP32 uniform u = k 2^-24.  Error budget of -ln(1-u): 1 - u exact;
    s = (m-1)/(m+1) carries two roundings (m+1 and the quotient, 1 ulp); the
    series tail is added to the exact 2s with its own error scaled by at most
    s^2/3 < 0.01; the two fma's of e ln2 add 0.5 ulp each of a dominant term.
    The bound taken is 2 ulp of the true value (the maximum seen is 1.65)."""
    e = O.transform(O.DIST_EXPONENTIAL, ALL_U.astype(np.float32))
    ref = -np.log1p(-ALL_U)
    assert e[0] == 0.0 and not np.signbit(e[0])
    assert ulp_err(e[1:], ref[1:]).max() <= 2.0
    assert np.all(np.diff(e) >= 0)      # monotone in u


@pytest.mark.parametrize("x,expect", [(1.0, 0.0), (0.5, -float(np.float32(float(LN2))))])
def test_ln_exact_points(x, expect):
    assert O.ln_unit_f32(x) == expect


def test_ln_powers_of_two():
    for k in range(1, 25):
        got = O.ln_unit_f32(2.0**-k)
        assert ulp_err(got, -k * math.log(2.0)) <= 1.0, k


def test_sincos_exhaustive_within_two_ulp():
    """Every FP32 uniform: sin and cos of 2 pi u against float64 libm.  With
    the reflection r -> 1 - r the polynomials see (pi/2) r <= pi/4, so both
    results keep a small relative error also next to their zeros; away from
    the exact zeros the bound is 2 ulp of the true value."""
    u32 = ALL_U.astype(np.float32)
    s, c = O.sincos_2pi_array(u32)
    t = 2.0 * np.pi * ALL_U
    sr, cr = np.sin(t), np.cos(t)
    exact_zero_s = (np.arange(1 << 24) % (1 << 23)) == 0        # u = 0, 1/2
    exact_zero_c = (np.arange(1 << 24) % (1 << 23)) == (1 << 22)  # u = 1/4, 3/4
    assert np.all(s[exact_zero_s] == 0) and np.all(c[exact_zero_c] == 0)
    assert ulp_err(s[~exact_zero_s], sr[~exact_zero_s]).max() <= 2.0
    assert ulp_err(c[~exact_zero_c], cr[~exact_zero_c]).max() <= 2.0
    assert np.all(np.abs(s) <= 1) and np.all(np.abs(c) <= 1)


@pytest.mark.parametrize("u,s,c", [(0.0, 0.0, 1.0), (0.25, 1.0, 0.0), (0.5, 0.0, -1.0), (0.75, -1.0, 0.0)])
def test_sincos_quadrant_points(u, s, c):
    assert O.sincos_2pi_f32(u) == (s, c)


def test_sincos_symmetries():
    """sin(2 pi (1/2 - u)) = sin(2 pi u) and cos(2 pi (1 - u)) = cos(2 pi u):
    the quadrant logic and the reflection must agree with each other."""
    k = np.arange(1, 1 << 22, 7, dtype=np.int64)
    u = (k * 2.0**-24).astype(np.float32)
    s1, c1 = O.sincos_2pi_array(u)
    s2, _ = O.sincos_2pi_array(((1 << 23) - k) * 2.0**-24)
    _, c3 = O.sincos_2pi_array(((1 << 24) - k) * 2.0**-24)
    assert np.array_equal(s1, s2)
    assert np.array_equal(c1, c3)


def _uniforms(n, seed=0xC0FFEE):
    return O.philox_generate((seed & 0xFFFFFFFF, seed >> 32), 0, 0, n, O.OUT_F32)


def test_normal_pairs_match_the_formula():
    u = _uniforms(1 << 20)
    z = O.transform(O.DIST_NORMAL, u).astype(np.float64)
    u0, u1 = u[0::2].astype(np.float64), u[1::2].astype(np.float64)
    r = np.sqrt(-2.0 * np.log1p(-u0))
    t = 2.0 * np.pi * u1
    # r within ~1.5 ulp, sin/cos within 2 ulp, one product rounding: 4 ulp of r
    tol = 4 * np.spacing(r.astype(np.float32)).astype(np.float64) + 1e-30
    assert np.all(np.abs(z[0::2] - r * np.cos(t)) <= tol)
    assert np.all(np.abs(z[1::2] - r * np.sin(t)) <= tol)


def test_distributions():
    """Moments and Kolmogorov-Smirnov distances of 2^21 variates from Philox
    uniforms (fixed seed; thresholds far outside sampling noise)."""
    stats = pytest.importorskip("scipy.stats")
    u = _uniforms(1 << 21)
    z = O.transform(O.DIST_NORMAL, u).astype(np.float64)
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs((z**4).mean() - 3) < 5 * math.sqrt(96 / n)
    assert stats.kstest(z, "norm").statistic < 1.63 * 1.5 / math.sqrt(n)
    # pairs are independent: correlation of the two halves of each pair
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5 / math.sqrt(n / 2)
    e = O.transform(O.DIST_EXPONENTIAL, u).astype(np.float64)
    assert abs(e.mean() - 1) < 5 / math.sqrt(n)
    assert abs(e.var() - 1) < 5 * math.sqrt(8 / n)
    assert stats.kstest(e, "expon").statistic < 1.63 * 1.5 / math.sqrt(n)


def test_odd_normal_length_is_rejected():
    with pytest.raises(ValueError):
        O.transform(O.DIST_NORMAL, np.zeros(3, dtype=np.float32))
