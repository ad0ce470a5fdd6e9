"""Deterministic sine and cosine for the sine-band refinement predicate (TEST
INFRASTRUCTURE).

The sine-band grids (Sec. 4.1 style narrow band around the zero set of a smooth random
field) decide refinement from sin and cos of the cell centre.  Two independent builders
can only produce the same octree if they evaluate those functions identically, so both
follow one published recipe rather than a platform libm:

  * Cody and Waite's additive range reduction (W. J. Cody, W. Waite, "Software Manual
    for the Elementary Functions", 1980): k = nearest integer to a * (2/pi),
    r = ((a - k P1) - k P2) - k P3 with pi/2 = P1 + P2 + P3, where P1 and P2 carry 33
    significant bits so that k * P1 and k * P2 are exact for |k| < 2^20;
  * Taylor series of sin and cos about 0 on |r| <= pi/4 (terms to r^17 and r^18; the
    first omitted term is below 1e-19), evaluated by Horner's rule from the highest
    term, coefficients (-1)^j / n! formed by one division of the exactly representable
    factorial;
  * the quadrant k mod 4 selects (sin r, cos r, -sin r, -cos r) for sin a and
    (cos r, -sin r, -cos r, sin r) for cos a.

Pinned in tests/test_oracle_trig.py against numpy's libm (a few ulp), exact special
values, sin^2 + cos^2 = 1, odd/even symmetry and the split of pi/2 recomputed in
300-bit arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

# pi/2 = P1 + P2 + P3 to about 1e-37 (P1, P2: 33 significant bits each)
P1 = float.fromhex("0x1.921fb544p+0")
P2 = float.fromhex("0x1.0b4611a6p-34")
P3 = float.fromhex("0x1.3198a2e037073p-69")
TWO_OVER_PI = float.fromhex("0x1.45f306dc9c883p-1")   # 2/pi rounded to double
TWO_PI = float.fromhex("0x1.921fb54442d18p+2")        # 2 pi rounded to double


def _coefficients():
    """sin: coefficients of r^3, r^5, ..., r^17; cos: of r^2, r^4, ..., r^18."""
    s, c = [], []
    for n in range(2, 19):
        sign = -1.0 if ((n // 2) % 2 == 1) else 1.0   # r^2, r^3: -; r^4, r^5: +; ...
        v = sign / float(math.factorial(n))
        (c if n % 2 == 0 else s).append(v)
    return s, c


SIN_C, COS_C = _coefficients()


def _reduce(a):
    a = np.asarray(a, np.float64)
    k = np.rint(a * TWO_OVER_PI)
    r = ((a - k * P1) - k * P2) - k * P3
    q = k.astype(np.int64) & 3
    return r, q


def _sin_r(r):
    r2 = r * r
    p = np.full(r.shape, SIN_C[-1])
    for c in SIN_C[-2::-1]:
        p = p * r2 + c
    return r + (r * r2) * p


def _cos_r(r):
    r2 = r * r
    p = np.full(r.shape, COS_C[-1])
    for c in COS_C[-2::-1]:
        p = p * r2 + c
    return 1.0 + r2 * p


def det_sin(a):
    r, q = _reduce(a)
    s, c = _sin_r(r), _cos_r(r)
    return np.select([q == 0, q == 1, q == 2], [s, c, -s], -c)


def det_cos(a):
    r, q = _reduce(a)
    s, c = _sin_r(r), _cos_r(r)
    return np.select([q == 0, q == 1, q == 2], [c, -s, -c], s)
