"""Pins of the oracle's deterministic sine and cosine (oracle/trig.py), the functions
the sine-band refinement predicate is built on, against libm, exact identities and
300-bit arithmetic."""
import math
from fractions import Fraction

import mpmath as mp
import numpy as np

from oracle import trig
from oracle import octree as O
from paper_2604_18886_b300 import problems as P


def test_pi_half_split_is_exact_to_1e_35():
    mp.mp.prec = 300
    s = mp.mpf(trig.P1) + mp.mpf(trig.P2) + mp.mpf(trig.P3)
    assert abs(s - mp.pi / 2) < mp.mpf(10) ** -35
    # the first two parts carry at most 33 significant bits, so k * P is exact for |k| < 2^20
    for p in (trig.P1, trig.P2):
        m, e = math.frexp(p)
        assert (m * 2 ** 33) == int(m * 2 ** 33)
    k = np.arange(-(2 ** 19), 2 ** 19, 977, dtype=np.float64)
    for p in (trig.P1, trig.P2):
        exact = [Fraction(int(v)) * Fraction(p) for v in k[:200]]
        assert all(Fraction(float(v * p)) == e for v, e in zip(k[:200], exact))


def test_taylor_coefficients_are_rounded_inverse_factorials():
    for j, c in enumerate(trig.SIN_C):
        n = 2 * j + 3
        assert c == float(Fraction((-1) ** (j + 1), math.factorial(n)))
    for j, c in enumerate(trig.COS_C):
        n = 2 * j + 2
        assert c == float(Fraction((-1) ** (j + 1), math.factorial(n)))


def test_agrees_with_libm_within_two_ulp():
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.uniform(-60, 60, 400000),
                        rng.uniform(-1e3, 1e3, 100000),
                        # around the quadrant boundaries k pi/4 where the reduction switches
                        (np.arange(-80, 81)[:, None] * (math.pi / 4) + np.linspace(-1e-9, 1e-9, 21)).ravel()])
    for f, g in ((trig.det_sin, np.sin), (trig.det_cos, np.cos)):
        err = np.abs(f(a) - g(a))
        assert err.max() <= 2.3e-16, err.max()


def test_high_precision_values():
    mp.mp.prec = 200
    a = np.random.default_rng(12).uniform(-50, 50, 300)
    s, c = trig.det_sin(a), trig.det_cos(a)
    for x, sv, cv in zip(a, s, c):
        assert abs(mp.mpf(sv) - mp.sin(mp.mpf(x))) < 2.3e-16
        assert abs(mp.mpf(cv) - mp.cos(mp.mpf(x))) < 2.3e-16


def test_identities_hold_exactly_or_to_rounding():
    a = np.random.default_rng(13).uniform(-40, 40, 100000)
    assert np.array_equal(trig.det_sin(-a), -trig.det_sin(a))      # odd, bit for bit
    assert np.array_equal(trig.det_cos(-a), trig.det_cos(a))       # even, bit for bit
    assert trig.det_sin(np.array([0.0]))[0] == 0.0 and trig.det_cos(np.array([0.0]))[0] == 1.0
    s, c = trig.det_sin(a), trig.det_cos(a)
    assert np.abs(s * s + c * c - 1.0).max() <= 6e-16
    # shift by a quarter period: sin(a + pi/2) = cos(a) up to the rounding of the argument
    assert np.abs(trig.det_sin(a + math.pi / 2) - c).max() <= 1e-14


def test_sine_band_predicate_matches_high_precision_evaluation():
    """The predicate's decisions equal those of the same formula in 200-bit arithmetic
    wherever the margin exceeds 1e-12 (brute force on a few thousand cell centres)."""
    p = P.sine_band(8, 3)
    d = p.desc
    rng = np.random.default_rng(14)
    depth = 2
    nd = d.n0 * 2 ** depth
    ijk = rng.integers(0, nd, size=(3000, 3))
    got = O.refine_predicate(d, depth, ijk[:, 0], ijk[:, 1], ijk[:, 2])
    mp.mp.prec = 200
    checked = 0
    for (i, j, k), g in zip(ijk, got):
        x = [(mp.mpf(int(v)) + mp.mpf(1) / 2) / nd for v in (i, j, k)]
        s = mp.mpf(0)
        gr = [mp.mpf(0)] * 3
        for (kap, dx, dy, dz, th) in d.sines:
            w = 2 * mp.pi * kap
            arg = w * (dx * x[0] + dy * x[1] + dz * x[2]) + th
            s += mp.sin(arg)
            gr = [gv + w * mp.cos(arg) * dv for gv, dv in zip(gr, (dx, dy, dz))]
        n = len(d.sines)
        phi = s / n
        gn = mp.sqrt(sum(v * v for v in gr)) / n
        margin = d.band + gn * mp.sqrt(3) / 2 / nd - abs(phi)
        if abs(margin) > 1e-12:
            assert bool(margin > 0) == bool(g)
            checked += 1
    assert checked > 2900
    assert 0 < got.sum() < len(got)
