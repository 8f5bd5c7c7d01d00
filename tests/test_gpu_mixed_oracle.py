"""The precision form's step decisions on the GPU against the oracle's own
precision-form tracker (orc_track_mixed, which restates the rules): on a
linear homotopy far from the thresholds the single-path tracker takes the
same steps and ends at the same point:

* a well-conditioned target (no rule fires): the same steps and the same end
  point;
* an integer 2 x 2 target with condition ~4.4e12 (the kappa_hat rule) and an
  integer triangular 3 x 3 target with unit pivots and off-diagonal 2^26 (the
  linear-contraction rule in the oracle): both trackers finish, and both
  escalate on the first.
"""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_END, cabs_diff, soa_from_complex
from paper_1501_06625_gb300 import libph, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    c.close()


def _case(name):
    if name == "well":
        rng = np.random.default_rng(3)
        A = rng.integers(-4, 5, (4, 4)).astype(float) + 8 * np.eye(4)
        xs = np.array([1 + 1j, 2 - 1j, -1, 1j])
    elif name == "kappa":
        a = float(2 ** 20)
        A = np.array([[a, a + 1], [a - 1, a]])
        xs = np.array([1 + 1j, 2 - 1j])
    else:
        M = float(2 ** 26)
        A = np.array([[1.0, M, M], [0.0, 1.0, M], [0.0, 0.0, 1.0]])
        xs = np.array([1 + 1j, 2 - 1j, -1])
    n = A.shape[0]
    b, b0 = A @ xs, A @ np.ones(n)
    rows = lambda rhs: [[(A[i, j], [(j, 1)]) for j in range(n) if A[i, j] != 0] + [(-rhs[i], [])]
                        for i in range(n)]
    return synth.build_system(n, n, rows(b)), synth.build_system(n, n, rows(b0)), xs


def _run(ctx, name):
    L = 2
    fsp, gsp, xs = _case(name)
    n = len(xs)
    x0 = soa_from_complex(np.ones(n), L)
    gam = soa_from_complex([np.exp(0.7j)], L).reshape(L, 2)
    params = synth.default_params(L, max_steps=500, lin_prec=1)
    f, g = ctx.load(fsp, L), ctx.load(gsp, L)
    x = np.zeros_like(x0)
    st, s, log = libph.ph_track_path(ctx.h, f, g, gam, x0, params, x, log_cap=600)
    so, xo, sto, logo = oracle.track_mixed(oracle.System(fsp, L), x0, gam, params,
                                           g=oracle.System(gsp, L))
    return (st, s, log, x), (so, sto, logo, xo), xs


def test_well_conditioned_decisions_match_the_oracle(ctx):
    (st, s, log, x), (so, sto, logo, xo), xs = _run(ctx, "well")
    assert st == libph.PH_OK and so == oracle.OK
    assert [(r["t"], r["accepted"]) for r in log] == [(r["t"], r["accepted"]) for r in logo]
    assert s["escalated"] == sto["escalated"] == 0 and s["wp_rest"] == sto["wp_rest"] == 0
    assert s["solves_f64"] > 0 and sto["solves_f64"] > 0
    assert cabs_diff(x, xo).max() <= TOL_END[2] * max(1.0, np.abs(xs).max())


@pytest.mark.parametrize("name", ["kappa", "tri"])
def test_ill_conditioned_outcomes_match_the_oracle(ctx, name):
    """Near the thresholds the double solves of the two implementations (the
    oracle's textbook MGS, the library's unnormalised one) round differently
    at kappa u_double, and so may the step decisions: both must finish."""
    (st, s, _, _), (so, sto, _, _), _ = _run(ctx, name)
    assert st == libph.PH_OK and so == oracle.OK
    if name == "kappa":
        assert s["escalated"] >= 1 and sto["escalated"] >= 1
