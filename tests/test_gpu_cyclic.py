"""GPU parity on the cyclic n-roots systems (Section 4.2, Eq. (10)).

* n = 8, 16, 24: values and Jacobians of f and of the homotopy against the
  oracle at random points, within 1e-28 (DD) / 1e-58 (QD) relative to the sum
  of the term magnitudes of each output;
* n = 128 and 352, where the oracle would take minutes: closed forms.  At the
  all-ones point f_i = n for i < n and f_n = 0, d f_i / d x_j = i (each variable
  lies in i of the n cyclic windows of length i) and d f_n / d x_j = 1: exact
  integers, which the GPU must return bit for bit.  At x_k = w^k (w = e^{2 pi i/n},
  built in 400-bit arithmetic and rounded to the working precision) f_i = 0 for
  i < n, so |f_i| must be within the tolerance times the n unit-modulus terms.
"""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_EVAL, assert_eval_close, soa_from_complex
from paper_1501_06625_gb300 import libph, synth

mpmath = pytest.importorskip("mpmath")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    c.close()


def _eval(ctx, L, f, n, x, t=1.0, gam=None, k=1):
    h = np.zeros((L, 2, n))
    J = np.zeros((L, 2, n, n))
    tl = np.zeros(L)
    tl[0] = t
    libph.ph_eval_jac(ctx.h, f, None, gam, k, tl, x, h, J)
    return h, J


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("n", [8, 16, 24])
def test_cyclic_parity_random_points(ctx, L, n):
    spec = synth.cyclic_system(n)
    rng = synth.Rng(300 + n)
    x = soa_from_complex(synth.random_x(rng, n), L)
    x[1] = x[0] * 2.0 ** -55                     # use the low limb too
    f = ctx.load(spec, L)
    of = oracle.System(spec, L)
    h, J = _eval(ctx, L, f, n, x, t=0.0)
    ho, Jo = oracle.eval_h(of, x)
    assert_eval_close(L, spec, x, h, J, ho, Jo)
    gam = soa_from_complex([rng.unit_complex()], L).reshape(L, 2)
    h, J = _eval(ctx, L, f, n, x, t=0.43, gam=gam)
    ho, Jo = oracle.eval_h(of, x, t=0.43, gamma=gam)
    assert_eval_close(L, spec, x, h, J, ho, Jo, t=0.43, gamma=gam, k=1)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("n", [128, 352])
def test_cyclic_closed_form_all_ones(ctx, L, n):
    spec = synth.cyclic_system(n)
    f = ctx.load(spec, L)
    x = soa_from_complex(np.ones(n), L)
    h, J = _eval(ctx, L, f, n, x, t=0.0)
    want_h = np.full(n, float(n))
    want_h[-1] = 0.0
    assert np.array_equal(h[0, 0], want_h) and not np.any(h[0, 1]) and not np.any(h[1:])
    want_J = np.tile(np.arange(1, n + 1, dtype=float), (n, 1))   # [col j][row i] = i + 1
    want_J[:, -1] = 1.0
    assert np.array_equal(J[0, 0], want_J) and not np.any(J[0, 1]) and not np.any(J[1:])


@pytest.mark.parametrize("L", [2, 4])
def test_cyclic_root_of_unity(ctx, L):
    n = 128
    mp = mpmath.mp
    mp.prec = 400
    from refmath import soa_from_mp
    w = [mp.exp(2j * mp.pi * k / n) for k in range(n)]
    x = soa_from_mp(w, L, mp)
    f = ctx.load(synth.cyclic_system(n), L)
    h, _ = _eval(ctx, L, f, n, x, t=0.0)
    mag = np.abs(h[0, 0, :-1] + 1j * h[0, 1, :-1])
    # each f_i is a sum of n products of unit modulus, rounded x_k: |f_i| is
    # the rounding of the inputs and of the sum, far below the tolerance
    assert mag.max() <= TOL_EVAL[L] * n, mag.max()


@pytest.mark.parametrize("L", [1, 2, 4])
def test_summation_lanes_tuned(ctx, L):
    """The summation's lanes per output are chosen by timing 1 .. 32 lanes (the
    paper's #Th); the choice is the fastest measured, and the evaluation with
    it still matches the oracle."""
    n = 16
    spec = synth.cyclic_system(n)
    f = ctx.load(spec, L)
    x = soa_from_complex(synth.random_x(synth.Rng(5), n), L)
    h, J = _eval(ctx, L, f, n, x, t=0.0)
    lanes, ms = libph.ph_sum_lanes(ctx.h, f)
    assert lanes in (1, 2, 4, 8, 16, 32)
    assert all(m > 0 for m in ms)
    assert ms[[1, 2, 4, 8, 16, 32].index(lanes)] == min(ms)
    ho, Jo = oracle.eval_h(oracle.System(spec, L), x)
    assert_eval_close(L, spec, x, h, J, ho, Jo)
