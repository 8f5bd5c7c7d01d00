"""Pins of the oracle's precision-form path tracker (orc_track_mixed: Newton
systems in double, residual and update in DD/QD, and the step rules of the
library's precision form) on cases that each exercise one rule, checked
against closed forms and against the oracle's all-working-precision tracker:

* a well-conditioned linear homotopy: no rule fires; the end point is the
  exact solution and the working-precision tracker's end point;
* an integer 2 x 2 target with condition ~4.4e12 and pivot ratio of the same
  size: the kappa_hat u_double > 1e-6 rule sends failed steps to working
  precision;
* an integer 3 x 3 upper-triangular target with unit pivots and off-diagonal
  2^26: the pivot ratio stays below 2 (kappa_hat u_double ~ 2e-16) while the
  condition is ~5e23, so the double corrector stops converging quadratically;
  only the linear-contraction rule sees it, and the rest of the path runs in
  working precision;
* an end game from the start: the tracker is the working-precision tracker,
  step for step and bit for bit.
"""
import numpy as np
import pytest

from paper_1501_06625_gb300 import synth

U_DD = 2.0 ** -104


def _soa(z, L):
    x = np.zeros((L, 2, len(z)))
    x[0, 0], x[0, 1] = np.real(z), np.imag(z)
    return x


def _linear_homotopy(orc, A, xs, L):
    """f = A x - b with b = A x*, g = A x - b0 with b0 = A 1 (exact for integer
    A and small integer x*), start x0 = 1."""
    n = A.shape[0]
    x0 = np.ones(n)
    b, b0 = A @ xs, A @ x0
    fsp = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n) if A[i, j] != 0]
                                    + [(-b[i], [])] for i in range(n)])
    gsp = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n) if A[i, j] != 0]
                                    + [(-b0[i], [])] for i in range(n)])
    gam = _soa([np.exp(0.7j)], L).reshape(L, 2)
    return orc.System(fsp, L), orc.System(gsp, L), _soa(x0.astype(complex), L), gam


def _lead(x):
    return x[0, 0] + 1j * x[0, 1]


def test_well_conditioned_path_no_rule(orc):
    L = 2
    rng = np.random.default_rng(3)
    A = rng.integers(-4, 5, (4, 4)).astype(float) + 8 * np.eye(4)
    xs = np.array([1 + 1j, 2 - 1j, -1, 1j])
    f, g, x0, gam = _linear_homotopy(orc, A, xs, L)
    p = synth.default_params(L, max_steps=500)
    st, x, stats, _ = orc.track_mixed(f, x0, gam, p, g=g)
    assert st == orc.OK
    assert stats["solves_f64"] > 0 and stats["escalated"] == 0 and stats["wp_rest"] == 0
    assert np.abs(_lead(x) - xs).max() < 1e-20
    st2, x2, _, _ = orc.track(f, x0, gam, p, g=g)
    assert st2 == orc.OK and np.abs(_lead(x) - _lead(x2)).max() < 1e-20


def test_kappa_rule_escalates(orc):
    L = 2
    a = float(2 ** 20)
    A = np.array([[a, a + 1], [a - 1, a]])
    xs = np.array([1 + 1j, 2 - 1j])
    f, g, x0, gam = _linear_homotopy(orc, A, xs, L)
    st, x, stats, _ = orc.track_mixed(f, x0, gam, synth.default_params(L, max_steps=500), g=g)
    assert st == orc.OK
    assert stats["escalated"] >= 1 and stats["cond"] * 2.0 ** -53 > 1e-6
    assert np.abs(_lead(x) - xs).max() < 1e3 * np.linalg.cond(A) * U_DD


def test_linear_contraction_rule_falls_back(orc):
    L = 2
    M = float(2 ** 26)
    A = np.array([[1.0, M, M], [0.0, 1.0, M], [0.0, 0.0, 1.0]])
    xs = np.array([1 + 1j, 2 - 1j, -1])
    f, g, x0, gam = _linear_homotopy(orc, A, xs, L)
    st, x, stats, _ = orc.track_mixed(f, x0, gam, synth.default_params(L, max_steps=500), g=g)
    assert st == orc.OK
    assert stats["cond"] * 2.0 ** -53 < 1e-12            # the pivot ratio sees nothing
    assert stats["wp_rest"] == 1 and stats["escalated"] >= 1
    # a triangular target with integer entries: the working-precision
    # corrector lands on the exact solution
    assert np.abs(_lead(x) - xs).max() < 1e-20


@pytest.mark.parametrize("L", [2, 4])
def test_end_game_from_the_start_is_the_plain_tracker(orc, L):
    rng = synth.Rng(21)
    spec = synth.dense_system(rng, 5, 5, 3, (1, 2))
    f = orc.System(spec, L)
    gam = _soa([rng.unit_complex()], L).reshape(L, 2)
    x0 = _soa(np.ones(5), L)
    p = synth.default_params(L, fixed_steps=20, max_newton=3)
    _, xp, sp, logp = orc.track(f, x0, gam, p)
    _, xm, sm, logm = orc.track_mixed(f, x0, gam, dict(p, endgame_t=1e-9))
    assert sm["solves_f64"] == 0 and logm == logp
    assert np.array_equal(xm, xp)
