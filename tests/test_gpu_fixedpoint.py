"""The fixed-point updates of the MGS kernels (ph_debug_update): a - ar b + sg
ai c for double-double operands (exact products of the leading limbs and the
cross products summed as 128-bit integers, exsum.cuh) and quad-double operands
(256-bit fixed-point values, products of their top words, qfx.cuh), checked
against exact rational arithmetic.

Bounds, relative to the terms' scale |a| + |ar b| + |ai c|: DD drops the
products of two trailing limbs (below 2^-106 of a product) and rounds the sum
of the cross products once in double (below 2^-105); the integer sum truncates
each term below 2^-124 of the largest.  QD converts each value exactly when its
limbs span fewer than 253 bits, drops partial products below 2^-240 of a
product, and truncates the sum below 2^-249 of the largest term.  On top of
these, the result is rounded to its limbs (half an ulp of the last).  The
tests use 2^-100 (DD) and 2^-230 (QD), plus that half ulp.  Cancellation to a
tiny result, zeros and a NaN operand are covered."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1501_06625_gb300 import libph

pytestmark = pytest.mark.gpu
TOL = {2: Fraction(2) ** -100, 4: Fraction(2) ** -230}


@pytest.fixture(scope="module")
def lib():
    from paper_1501_06625_gb300 import build
    build.build()
    return libph


def _normalised(rng, L, scale):
    """A multi-limb value: each limb below half an ulp of the one before."""
    v = np.zeros(L)
    v[0] = rng.standard_normal() * scale
    for l in range(1, L):
        v[l] = v[l - 1] * 2.0 ** -53 * (rng.random() - 0.5)
    return v


def _exact(v):
    return sum(Fraction(float(x)) for x in v)


def _to_limbs(x: Fraction, L):
    """The limbs of an exact value: each the nearest double to what remains."""
    out = []
    for _ in range(L):
        d = float(x)
        out.append(d)
        x -= Fraction(d)
    return np.array(out)


def _check(cases, got):
    L = cases.shape[2]
    for c in range(cases.shape[0]):
        a, ar, b, ai, cc, sgv = (cases[c, q] for q in range(6))
        sg = -1 if sgv[0] < 0 else 1
        exact = _exact(a) - _exact(ar) * _exact(b) + sg * _exact(ai) * _exact(cc)
        scale = abs(_exact(a)) + abs(_exact(ar) * _exact(b)) + abs(_exact(ai) * _exact(cc))
        out = got[c]
        for l in range(1, L):
            if out[l - 1] != 0.0:
                assert abs(out[l]) <= math.ulp(out[l - 1]) / 2, (c, out)
        tol = TOL[L] * scale
        if out[-1] != 0.0:
            tol += Fraction(math.ulp(out[-1])) / 2
        err = abs(_exact(out) - exact)
        assert err <= tol, (c, float(err), float(tol))


def _random_cases(rng, L, count):
    cases = np.zeros((count, 6, L))
    for c in range(count):
        for q in range(5):
            cases[c, q] = _normalised(rng, L, 10.0 ** rng.integers(-6, 6))
        cases[c, 5, 0] = 1.0 if c % 2 == 0 else -1.0
    return cases


@pytest.mark.parametrize("L", [2, 4])
def test_random_updates_against_exact_arithmetic(lib, L):
    rng = np.random.default_rng(40 + L)
    cases = _random_cases(rng, L, 400)
    _check(cases, lib.ph_debug_update(0, cases))


@pytest.mark.parametrize("L", [2, 4])
def test_cancellation_to_a_tiny_result(lib, L):
    """a set to the limbs of ar b - sg ai c (exactly rounded), plus a tiny
    perturbation in its last limb: the result is the perturbation, far below
    the terms' scale."""
    rng = np.random.default_rng(70 + L)
    cases = _random_cases(rng, L, 100)
    for c in range(cases.shape[0]):
        ar, b, ai, cc = (cases[c, q] for q in (1, 2, 3, 4))
        sg = -1 if cases[c, 5, 0] < 0 else 1
        v = _exact(ar) * _exact(b) - sg * _exact(ai) * _exact(cc)
        cases[c, 0] = _to_limbs(v, L)
        cases[c, 0, L - 1] += math.ulp(cases[c, 0, L - 1]) * 3
    _check(cases, lib.ph_debug_update(0, cases))


@pytest.mark.parametrize("L", [2, 4])
def test_zeros_and_nan(lib, L):
    rng = np.random.default_rng(5)
    cases = np.zeros((4, 6, L))
    cases[:, 5, 0] = 1.0
    cases[1, 0] = _normalised(rng, L, 2.0)            # a alone
    cases[2, 1] = _normalised(rng, L, 2.0)            # ar b with b = 0
    cases[2, 3] = _normalised(rng, L, 1.0)
    cases[2, 4] = _normalised(rng, L, 3.0)            # ai c alone
    cases[3] = cases[2]
    cases[3, 2, 0] = np.nan
    got = lib.ph_debug_update(0, cases)
    assert np.all(got[0] == 0.0)
    assert np.array_equal(got[1], cases[1, 0])
    _check(cases[:3], got[:3])
    assert not np.isfinite(got[3, 0])
