"""GPU parity of the precision form (lin_prec 1) in the single-path tracker,
whose step graph holds the working-precision and the double kernel sets and
gates one of them off per iteration:

* one mixed corrector iteration equals the oracle's (orc_newton_mixed) within
  the forward error bound of the double solve;
* a fixed schedule ends where the oracle's all-working-precision tracker ends,
  with every solve before the end game in double;
* an adaptive mixed path ends where the oracle's replay of its own schedule
  ends, which is the planted root, and takes the same steps as the many-path
  form;
* a target whose Jacobian has condition ~4e12 (kappa u_double above the
  escalation threshold) makes the double corrector fail and the step be
  corrected again in working precision, in both forms; the path still ends
  on the exact root;
* a fixed schedule with no Newton steps in double (end game from t = 0) is
  the plain tracker.
"""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_END, cabs_diff, lead_complex, soa_from_complex
from paper_1501_06625_gb300 import libph, synth
from test_gpu_mixed import planted_case, track1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    c.close()


def path1(ctx, f, gam, x0, params, g=None, log_cap=0):
    x = np.zeros_like(x0)
    st, stats, log = libph.ph_track_path(ctx.h, f, g, gam, x0, params, x, log_cap=log_cap)
    return st, x, stats, log


@pytest.mark.parametrize("L", [2, 4])
def test_one_mixed_iteration_matches_oracle(ctx, L):
    rng = synth.Rng(21)
    n = 7
    spec = synth.dense_system(rng, n, n, 3, (1, 2))
    gam = soa_from_complex([rng.unit_complex()], L).reshape(L, 2)
    x0 = soa_from_complex(synth.random_x(rng, n), L)
    params = synth.default_params(L, fixed_steps=1, max_newton=1, lin_prec=1, endgame_t=2.0)
    f = ctx.load(spec, L)
    st, x1, stats, _ = path1(ctx, f, gam, x0, params)
    assert st == libph.PH_OK and stats["updates"] == 1 and stats["solves_f64"] == 1
    of = oracle.System(spec, L)
    _, xr, _, _, _, _, _ = oracle.newton_mixed(of, x0, 1.0, gam, params, "f64", fixed=True)
    _, J = oracle.eval_h(of, x0, t=1.0, gamma=gam)
    kappa = np.linalg.cond((J[0, 0] + 1j * J[0, 1]).T)
    d = np.abs(lead_complex(xr) - lead_complex(x0)).max()
    err = cabs_diff(x1, xr).max()
    assert err <= 100 * n * kappa * 2.0 ** -53 * d + 10 * TOL_END[L], (err, kappa, d)
    assert 1.0 <= stats["cond"] <= kappa * 1.01


@pytest.mark.parametrize("L", [2, 4])
def test_fixed_schedule_endpoint(ctx, L):
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, fixed_steps=100, max_newton=3)
    st, x, stats, _ = path1(ctx, f, gam, start, dict(params, lin_prec=1))
    assert st == libph.PH_OK and stats["steps"] == 100
    assert stats["solves_f64"] == 99 * 3 and stats["escalated"] == 0
    _, xr, _, _ = oracle.track(of, start, gam, params)
    assert np.abs(lead_complex(xr) - xs).max() < 1e-20
    assert cabs_diff(x, xr).max() <= TOL_END[L]


@pytest.mark.parametrize("L", [2, 4])
def test_adaptive_replay_and_many_path_form(ctx, L):
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, max_steps=2000, max_newton=8, lin_prec=1)
    st, x, stats, log = path1(ctx, f, gam, start, params, log_cap=2100)
    assert st == libph.PH_OK, stats
    assert len(log) == stats["steps"] and stats["solves_f64"] > 0
    xr = oracle.replay(of, start, gam, params, log)
    assert cabs_diff(x, xr).max() <= TOL_END[L]
    assert np.abs(lead_complex(x) - xs).max() < 1e-20
    # the many-path form follows the same rules: the same schedule and end point
    xb, sb, logb = track1(ctx, f, gam, start, params, log_cap=2100)
    assert sb["status"] == libph.PH_OK
    assert [r["t"] for r in logb] == [r["t"] for r in log]
    assert (sb["accepted"], sb["escalated"]) == (stats["accepted"], stats["escalated"])
    assert cabs_diff(xb, x).max() <= TOL_END[L]


def _ill_conditioned(L):
    """f = A x - b and g = A x - b0 with the integer matrix
    A = [[2^20, 2^20 + 1], [2^20 - 1, 2^20]] (det 1, condition ~4.4e12):
    every coefficient and both roots (x* = (1+i, 2-i), x0 = (1, 1)) are exact,
    and J(t) = (gamma (1-t) + t) A for every t."""
    a = float(2 ** 20)
    A = np.array([[a, a + 1], [a - 1, a]])
    xs = np.array([1 + 1j, 2 - 1j])
    x0 = np.array([1.0 + 0j, 1.0 + 0j])
    b, b0 = A @ xs, A @ x0
    fsp = synth.build_system(2, 2, [[(A[i, 0], [(0, 1)]), (A[i, 1], [(1, 1)]), (-b[i], [])]
                                    for i in range(2)])
    gsp = synth.build_system(2, 2, [[(A[i, 0], [(0, 1)]), (A[i, 1], [(1, 1)]), (-b0[i], [])]
                                    for i in range(2)])
    return fsp, gsp, xs, soa_from_complex(x0, L), np.linalg.cond(A)


def test_escalation_to_working_precision(ctx):
    L = 2
    fsp, gsp, xs, x0, kappa = _ill_conditioned(L)
    f, g = ctx.load(fsp, L), ctx.load(gsp, L)
    gam = soa_from_complex([np.exp(0.7j)], L).reshape(L, 2)
    params = synth.default_params(L, max_steps=500, max_newton=3, lin_prec=1)
    st, x, stats, _ = path1(ctx, f, gam, x0, params, g=g)
    assert st == libph.PH_OK, stats
    assert stats["escalated"] >= 1 and stats["solves_f64"] >= 1
    assert stats["cond"] * 2.0 ** -53 > 1e-6            # above the escalation threshold
    err = np.abs(lead_complex(x) - xs).max()
    assert err <= 1e3 * kappa * 2.0 ** -106, err
    # the many-path form escalates the same steps
    xo = np.zeros((1,) + x0.shape)
    sb, _ = libph.ph_track_paths(ctx.h, f, g, gam, np.ascontiguousarray(x0[None]), params, xo)
    assert sb[0]["status"] == libph.PH_OK
    assert (sb[0]["steps"], sb[0]["escalated"]) == (stats["steps"], stats["escalated"])
    assert np.abs(lead_complex(xo[0]) - xs).max() <= 1e3 * kappa * 2.0 ** -106


@pytest.mark.parametrize("L", [2, 4])
def test_end_game_from_the_start_is_the_plain_tracker(ctx, L):
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, fixed_steps=40, max_newton=3)
    _, xp, sp, _ = path1(ctx, f, gam, start, params)
    _, xm, sm, _ = path1(ctx, f, gam, start, dict(params, lin_prec=1, endgame_t=1e-9))
    assert sm["solves_f64"] == 0 and sm["updates"] == sp["updates"]
    assert np.array_equal(xm, xp)
