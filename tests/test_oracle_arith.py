"""Pins of the oracle's multi-limb arithmetic against exact rational arithmetic.

Every oracle operation is the exact result rounded once to L limbs, so its
error relative to the exact result is at most about u^L (u = 2^-53).  These
tests compute the exact result with Python's fractions on random operands whose
leading exponents span +-300 (+-150 for products and quotients) and require the
relative error to stay below 2 u^L, the limbs to come out normalized, and the
two error-free transformations to be exact.  A dropped limb product, a wrong
sign or a mis-normalised limb shows up as an error near u, far above the bound.
"""
from fractions import Fraction

import numpy as np
import pytest

from refmath import U, frac_real, normalized, rand_limbs, rel_err

NSAMP = 1500


def _fr(col):
    return frac_real(col)


@pytest.mark.parametrize("L", [2, 4])
def test_round_sum_exact_then_rounded(orc, L):
    rng = np.random.default_rng(11 + L)
    for trial in range(400):
        m = int(rng.integers(1, 40))
        terms = rng.uniform(-1, 1, m) * np.exp2(rng.integers(-200, 200, m))
        if trial % 5 == 0:                     # heavy cancellation
            terms = np.concatenate([terms, -terms[: m // 2] * (1 + 2.0 ** -40)])
        exact = sum((Fraction(float(t)) for t in terms), Fraction(0))
        out = orc.round_sum(terms, L)
        assert normalized(out)
        assert rel_err(_fr(out), exact) <= 2 * U ** L


@pytest.mark.parametrize("L", [2, 4])
def test_error_free_transforms(orc, L):
    rng = np.random.default_rng(3)
    x = rand_limbs(rng, L, NSAMP, -300, 300)
    y = rand_limbs(rng, L, NSAMP, -300, 300)
    s = orc.vec_real("two_sum", L, x, y)
    for i in range(NSAMP):
        assert Fraction(s[0, i]) + Fraction(s[1, i]) == Fraction(x[0, i]) + Fraction(y[0, i])
        assert s[0, i] == x[0, i] + y[0, i]
    x = rand_limbs(rng, L, NSAMP, -150, 150)
    y = rand_limbs(rng, L, NSAMP, -150, 150)
    p = orc.vec_real("two_prod", L, x, y)
    for i in range(NSAMP):
        assert Fraction(p[0, i]) + Fraction(p[1, i]) == Fraction(x[0, i]) * Fraction(y[0, i])


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_real_ops_vs_fractions(orc, L, op):
    rng = np.random.default_rng(hash((L, op)) % 2**32)
    span = 300 if op in ("add", "sub") else 150
    x = rand_limbs(rng, L, NSAMP, -span, span)
    y = rand_limbs(rng, L, NSAMP, -span, span)
    if op in ("add", "sub"):                   # a share of near-cancellations
        k = NSAMP // 4
        y[:, :k] = -x[:, :k] if op == "add" else x[:, :k]
        y[L - 1, :k] += x[0, :k] * U ** L * rng.uniform(-4, 4, k)
    z = orc.vec_real(op, L, x, y)
    for i in range(NSAMP):
        a, b = _fr(x[:, i]), _fr(y[:, i])
        exact = {"add": a + b, "sub": a - b, "mul": a * b, "div": a / b}[op]
        assert normalized(z[:, i])
        assert rel_err(_fr(z[:, i]), exact) <= 2 * U ** L, (op, i)


@pytest.mark.parametrize("L", [2, 4])
def test_sqrt_vs_fractions(orc, L):
    rng = np.random.default_rng(5 + L)
    x = np.abs(rand_limbs(rng, L, NSAMP, -300, 300))
    x[1:] *= np.sign(x[0])
    z = orc.vec_real("sqrt", L, x)
    for i in range(NSAMP):
        a, s = _fr(x[:, i]), _fr(z[:, i])
        # |s - sqrt(a)| = |s^2 - a| / (s + sqrt(a)) ~ |s^2 - a| / (2 s)
        err = abs(s * s - a) / (2 * s * s)
        assert normalized(z[:, i])
        assert float(err) <= 3 * U ** L


@pytest.mark.parametrize("L", [2, 4])
def test_complex_ops_vs_fractions(orc, L):
    rng = np.random.default_rng(21 + L)
    n = NSAMP // 2
    x = np.stack([rand_limbs(rng, L, n, -100, 100), rand_limbs(rng, L, n, -100, 100)], axis=1)
    y = np.stack([rand_limbs(rng, L, n, -100, 100), rand_limbs(rng, L, n, -100, 100)], axis=1)
    mul = orc.vec_cplx("mul", L, x, y)
    cmul = orc.vec_cplx("conj_mul", L, x, y)
    add = orc.vec_cplx("add", L, x, y)
    ab2 = orc.vec_cplx("abs2", L, x)
    for i in range(n):
        ar, ai = _fr(x[:, 0, i]), _fr(x[:, 1, i])
        br, bi = _fr(y[:, 0, i]), _fr(y[:, 1, i])
        checks = [(mul[:, 0, i], ar * br - ai * bi), (mul[:, 1, i], ar * bi + ai * br),
                  (cmul[:, 0, i], ar * br + ai * bi), (cmul[:, 1, i], ar * bi - ai * br),
                  (add[:, 0, i], ar + br), (add[:, 1, i], ai + bi), (ab2[:, i], ar * ar + ai * ai)]
        for got, exact in checks:
            assert normalized(got)
            assert rel_err(_fr(got), exact) <= 2 * U ** L


def test_special_values(orc):
    # exact cancellation gives an exact zero; x - x = 0; 1/1 = 1; sqrt(4) = 2
    for L in (2, 4):
        one = np.zeros((L, 1)); one[0, 0] = 1.0
        four = np.zeros((L, 1)); four[0, 0] = 4.0
        third = orc.vec_real("div", L, one, 3 * one)
        assert _fr(orc.vec_real("sub", L, third, third)[:, 0]) == 0
        assert _fr(orc.vec_real("div", L, one, one)[:, 0]) == 1
        assert _fr(orc.vec_real("sqrt", L, four)[:, 0]) == 2
        # 3 * (1/3) differs from 1 by at most one rounding of L limbs
        back = orc.vec_real("mul", L, third, 3 * one)
        assert rel_err(_fr(back[:, 0]), Fraction(1)) <= 3 * U ** L
