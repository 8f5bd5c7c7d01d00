"""The oracle in complex double (one limb): every operation is the exact
result rounded once to a double, which is what IEEE double arithmetic
returns; so add, sub, mul, div and sqrt must equal Python's float operations
bit for bit, and a linear solve must match LAPACK to its error bound."""
import math

import numpy as np
import pytest

from paper_1501_06625_gb300 import synth
from refmath import soa_from_complex


def _operands(rng, count):
    a = rng.uniform(0.5, 1.0, count) * np.exp2(rng.integers(-300, 300, count)) * rng.choice([-1, 1], count)
    b = rng.uniform(0.5, 1.0, count) * np.exp2(rng.integers(-300, 300, count)) * rng.choice([-1, 1], count)
    return a, b


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_double_ops_are_ieee(orc, op):
    rng = np.random.default_rng(11)
    a, b = _operands(rng, 4000)
    z = orc.vec_real(op, 1, a[None], b[None])[0]
    ref = {"add": a + b, "sub": a - b, "mul": a * b, "div": a / b}[op]
    assert np.array_equal(z, ref)


def test_double_sqrt_is_ieee(orc):
    rng = np.random.default_rng(12)
    a = np.abs(_operands(rng, 4000)[0])
    z = orc.vec_real("sqrt", 1, a[None])[0]
    assert np.array_equal(z, np.sqrt(a))


def test_double_solve_against_lapack(orc):
    rng = np.random.default_rng(13)
    n = 9
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    J = np.zeros((1, 2, n, n))
    J[0, 0], J[0, 1] = A.real.T, A.imag.T
    st, dx, rn = orc.mgs_solve(J, soa_from_complex(b, 1))
    assert st == orc.OK
    x = dx[0, 0] + 1j * dx[0, 1]
    ref = np.linalg.solve(A, b)
    assert np.abs(x - ref).max() <= 100 * n * np.linalg.cond(A) * 2.0 ** -53 * np.abs(ref).max()


def test_double_eval_matches_float_arithmetic(orc):
    """x^3 - c at a double point: the oracle rounds each operation once, as
    Python's floats do in the same order."""
    c = 0.3 + 0.4j
    spec = synth.build_system(1, 1, [[(1.0, [(0, 3)]), (-c, [])]])
    f = orc.System(spec, 1)
    x = 0.7 - 0.2j
    h, J = orc.eval_h(f, soa_from_complex([x], 1))
    want = x * x * x - c
    assert abs(complex(h[0, 0, 0], h[0, 1, 0]) - want) <= 4 * 2.0 ** -53 * (abs(x) ** 3 + abs(c))
    assert abs(complex(J[0, 0, 0, 0], J[0, 1, 0, 0]) - 3 * x * x) <= 8 * 2.0 ** -53 * 3 * abs(x) ** 2
