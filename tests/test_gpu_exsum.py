"""The exact warp sum the MGS kernels use for their dot products and norms
(exsum.cuh, through ph_debug_warp_sum): 32 double-double or quad-double values
summed as fixed-point integers and rounded back limb by limb, checked against
exact rational sums: the limbs are normalised (each within half an ulp of the
one before), and their sum equals the exact sum of the inputs within the
truncation bound 32 * 2^(e + 59 - 64 W) (e the exponent of the last bit of the
largest leading limb, W = 2 for DD, 4 for QD) plus half an ulp of the last
limb.  Cancellation to zero, zeros and a NaN input are covered."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1501_06625_gb300 import libph

pytestmark = pytest.mark.gpu
W = {2: 2, 4: 4}


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


def _check(lib, vals):
    L = vals.shape[1]
    out = lib.ph_debug_warp_sum(0, vals)
    exact = sum(Fraction(float(x)) for x in vals.reshape(-1))
    lead = [x for x in vals[:, 0] if x != 0.0]
    if not lead:
        assert np.all(out == 0.0)
        return
    e = max(math.frexp(abs(x))[1] - 53 for x in lead)     # exponent of the last bit
    base = e + 59 - 64 * W[L]
    for l in range(1, L):
        if out[l - 1] != 0.0:
            assert abs(out[l]) <= math.ulp(out[l - 1]) / 2
    got = sum(Fraction(float(x)) for x in out)
    tol = 32 * Fraction(2) ** base + Fraction(math.ulp(out[-1])) / 2 if out[-1] else \
        32 * Fraction(2) ** base
    assert abs(got - exact) <= tol, (float(got - exact), float(tol))


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("case", range(8))
def test_random_values_with_spread_exponents(lib, L, case):
    rng = np.random.default_rng(case * 7 + L)
    vals = np.stack([_normalised(rng, L, 10.0 ** rng.integers(-12, 12)) for _ in range(32)])
    _check(lib, vals)


@pytest.mark.parametrize("L", [2, 4])
def test_cancellation(lib, L):
    rng = np.random.default_rng(99 + L)
    half = np.stack([_normalised(rng, L, 1.0) for _ in range(16)])
    vals = np.concatenate([half, -half[::-1]])          # sums to exactly zero
    assert np.all(lib.ph_debug_warp_sum(0, vals) == 0.0)
    vals[5, -1] += 2.0 ** -200                           # all but one tiny limb cancels
    _check(lib, vals)


@pytest.mark.parametrize("L", [2, 4])
def test_zeros_single_value_and_nan(lib, L):
    vals = np.zeros((32, L))
    assert np.all(lib.ph_debug_warp_sum(0, vals) == 0.0)
    rng = np.random.default_rng(5)
    vals[17] = _normalised(rng, L, 3.0)
    out = lib.ph_debug_warp_sum(0, vals)
    assert out[0] == vals[17, 0]                         # one value: its leading limb unchanged
    _check(lib, vals)
    vals[3, 0] = np.nan
    assert np.all(np.isnan(lib.ph_debug_warp_sum(0, vals)))
