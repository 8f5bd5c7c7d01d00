"""GPU parity of the precision form (lin_prec != 0): the Newton system in IEEE
double or single, the residual and the update in double-double/quad-double.

* one mixed corrector iteration equals the oracle's (orc_newton_mixed) within
  the forward error bound of the low-precision solve, in double and single;
* a fixed schedule ends where the oracle's all-working-precision tracker ends
  (the end game at t = 1 runs in working precision), in DD and QD;
* adaptive mixed paths end where the oracle's replay of their own schedule ends;
* the automatic choice takes single precision once the condition estimate
  allows it, never when the threshold is below 1, and reports its counts;
* the planted root of a system with coefficient moduli up to 1e12 is recovered
  by tracking it back to its start root and forward again in mixed precision;
* the serving loop gives the many-path form's result for a mixed job.
"""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_END, cabs_diff, lead_complex, soa_from_complex
from paper_1501_06625_gb300 import libph, synth

pytestmark = pytest.mark.gpu

U = {1: 2.0 ** -53, 2: 2.0 ** -24}


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    c.close()


def track1(ctx, f, gam, x0, params, log_cap=0):
    xo = np.zeros((1,) + x0.shape)
    stats, logs = libph.ph_track_paths(ctx.h, f, None, gam, np.ascontiguousarray(x0[None]),
                                       params, xo, log_cap=log_cap)
    return xo[0], stats[0], logs[0] if log_cap else None


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("lin", [1, 2])
def test_one_mixed_iteration_matches_oracle(ctx, L, lin):
    rng = synth.Rng(21)
    n = 7
    spec = synth.dense_system(rng, n, n, 3, (1, 2))
    g = rng.unit_complex()
    gam = soa_from_complex([g], L).reshape(L, 2)
    x0 = soa_from_complex(synth.random_x(rng, n), L)
    # one step from t = 0 straight to t = 1: the predictor returns x0, then one
    # corrector iteration at t = 1 (no end game)
    params = synth.default_params(L, fixed_steps=1, max_newton=1, lin_prec=lin, endgame_t=2.0)
    f = ctx.load(spec, L)
    x1, st, _ = track1(ctx, f, gam, x0, params)
    assert st["status"] == libph.PH_OK and st["updates"] == 1
    assert st["solves_f64" if lin == 1 else "solves_f32"] == 1
    of = oracle.System(spec, L)
    _, xr, it, upd, res, dxn, cond = oracle.newton_mixed(of, x0, 1.0, gam, params,
                                                         "f64" if lin == 1 else "f32", fixed=True)
    h, J = oracle.eval_h(of, x0, t=1.0, gamma=gam)
    Jc = J[0, 0] + 1j * J[0, 1]                    # leading limbs, [col][row]
    kappa = np.linalg.cond(Jc.T)
    d = np.abs(lead_complex(xr) - lead_complex(x0)).max()
    err = cabs_diff(x1, xr).max()
    assert err <= 100 * n * kappa * U[lin] * d + 10 * TOL_END[L], (err, kappa, d)
    # the condition estimate is a lower bound of the condition number
    assert 1.0 <= st["cond"] <= kappa * 1.01


_PLANTED = {}


def planted_case(L):
    """A planted system (n = 6, 6 terms over 3 variables, exponents {1,2}) and
    the start root of its planted root's path, found by the oracle tracking x*
    backwards (the homotopy with f and g swapped and 1/gamma), rounded to the
    exact root of unity it approaches."""
    if L not in _PLANTED:
        n = 6
        rng = synth.Rng(5)
        spec, xs = synth.planted_system(rng, n, n, 3, (1, 2), 0.0)
        d = spec.degrees()
        gsp = synth.build_system(n, n, [[(1.0, [(i, int(d[i]))]), (-1.0, [])] for i in range(n)])
        g = rng.unit_complex()
        gam = soa_from_complex([g], L).reshape(L, 2)
        gi = soa_from_complex([1.0 / g], L).reshape(L, 2)
        of, og = oracle.System(spec, L), oracle.System(gsp, L)
        st, xb, _, _ = oracle.track(og, soa_from_complex(xs, L), gi, synth.default_params(L), g=of)
        assert st == oracle.OK
        z = lead_complex(xb)
        start = np.exp(2j * np.pi * np.round(np.angle(z) * d / (2 * np.pi)) / d)
        _PLANTED[L] = (spec, xs, gam, soa_from_complex(start, L), of)
    return _PLANTED[L]


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("lin", [1, 2, 3])
def test_fixed_schedule_endpoint(ctx, L, lin):
    """100 fixed steps with 3 updates each along the planted root's path: the
    mixed-precision end point equals the oracle's all-working-precision end
    point (the last step, at t = 1, is the working-precision end game)."""
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, fixed_steps=100, max_newton=3)
    x, st, _ = track1(ctx, f, gam, start, dict(params, lin_prec=lin))
    assert st["status"] == libph.PH_OK and st["steps"] == 100
    assert st["solves_f64"] + st["solves_f32"] == 99 * 3        # all but the end game
    _, xr, _, _ = oracle.track(of, start, gam, params)
    assert np.abs(lead_complex(xr) - xs).max() < 1e-20            # the path converges
    err = cabs_diff(x, xr).max()
    assert err <= TOL_END[L], err


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("lin", [1, 3])
def test_adaptive_mixed_replay(ctx, L, lin):
    """Adaptive steps along the planted root's path in mixed precision: the
    oracle replays the GPU's own schedule in working precision and ends at the
    same point, which is x*."""
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, max_steps=2000, max_newton=8, lin_prec=lin)
    x, st, log = track1(ctx, f, gam, start, params, log_cap=2100)
    assert st["status"] == libph.PH_OK, st
    assert len(log) == st["steps"]
    xr = oracle.replay(of, start, gam, params, log)
    err = cabs_diff(x, xr).max()
    assert err <= TOL_END[L], err
    assert np.abs(lead_complex(x) - xs).max() < 1e-20


def test_auto_precision_choice(ctx):
    L = 2
    wl = synth.dense8(3, "dd")
    f = ctx.load(wl.f, L)
    base = dict(wl.params, fixed_steps=20, max_newton=3)
    _, st, _ = track1(ctx, f, wl.gamma_soa(), wl.x0_soa(), dict(base, lin_prec=3, cond_f32=1e8))
    assert st["solves_f32"] > 0 and st["solves_f64"] >= 1      # the first solve is in double
    assert st["cond"] >= 1.0
    _, st, _ = track1(ctx, f, wl.gamma_soa(), wl.x0_soa(), dict(base, lin_prec=3, cond_f32=0.5))
    assert st["solves_f32"] == 0 and st["solves_f64"] == 19 * 3
    _, st, _ = track1(ctx, f, wl.gamma_soa(), wl.x0_soa(), dict(base, lin_prec=0))
    assert st["solves_f32"] == 0 and st["solves_f64"] == 0


@pytest.mark.parametrize("L", [2, 4])
def test_planted_root_recovered(ctx, L):
    """Track the planted root x* back to its start root (the homotopy with the
    roles of f and g swapped and 1/gamma: the same curve), then forward in mixed
    precision; the end point is x* (which satisfies f(x*) = 0 exactly)."""
    n = 8
    rng = synth.Rng(77)
    spec, xs = synth.planted_system(rng, n, n, 4, (1, 2), 12.0)
    d = spec.degrees()
    gsp = synth.build_system(n, n, [[(1.0, [(i, int(d[i]))]), (-1.0, [])] for i in range(n)])
    g = rng.unit_complex()
    f = ctx.load(spec, L)
    gs = ctx.load(gsp, L)
    gam = soa_from_complex([g], L).reshape(L, 2)
    gam_inv = soa_from_complex([1.0 / g], L).reshape(L, 2)
    xstar = soa_from_complex(xs, L)
    params = synth.default_params(L, max_steps=2000, max_newton=8, lin_prec=1)
    # backwards: gamma' (1-s) f + s g from x* at s = 0
    xb = np.zeros((1,) + xstar.shape)
    sb, _ = libph.ph_track_paths(ctx.h, gs, f, gam_inv, np.ascontiguousarray(xstar[None]),
                                 params, xb)
    assert sb[0]["status"] == libph.PH_OK, sb[0]
    z = lead_complex(xb[0])
    assert np.abs(np.abs(z) - 1.0).max() < 1e-12         # a root of x_i^{d_i} = 1
    start = soa_from_complex(np.exp(2j * np.pi * np.round(np.angle(z) * d / (2 * np.pi)) / d), L)
    # forwards from that start root, total-degree homotopy, mixed precision
    x, st, _ = track1(ctx, f, gam, start, params)
    assert st["status"] == libph.PH_OK, st
    # x* is exact; the end point is within the corrector's tolerance of it,
    # or within kappa u_L where the Jacobian at x* is ill-conditioned
    _, J = oracle.eval_h(oracle.System(spec, L), xstar, t=1.0)
    kappa = np.linalg.cond((J[0, 0] + 1j * J[0, 1]).T)
    err = cabs_diff(x, xstar).max()
    assert err <= 1e3 * kappa * 2.0 ** (-53 * L) + 10 * params["tol_dx"], (err, kappa)


def test_serving_mixed_job_equals_many_path_form(ctx):
    L = 2
    rng = synth.Rng(8)
    spec = synth.dense_system(rng, 9, 9, 3, (1, 2))
    f = ctx.load(spec, L)
    gam = soa_from_complex([rng.unit_complex()], L).reshape(L, 2)
    x0 = soa_from_complex(np.ones(9), L)
    params = synth.default_params(L, max_steps=29, lin_prec=3)
    srv = libph.ph_server_create(ctx.h, max_n=16, pool_bytes=1 << 26, queue_cap=8)
    try:
        jid = libph.ph_server_submit(ctx.h, srv, f, None, gam, x0, params)
        xs = np.zeros_like(x0)
        ss, _ = libph.ph_server_wait(ctx.h, srv, jid, 60000, xs)
    finally:
        libph.ph_server_destroy(srv)
    xb, sb, _ = track1(ctx, f, gam, x0, params)
    assert np.array_equal(xs, xb)
    assert ss["solves_f32"] == sb["solves_f32"] and ss["solves_f64"] == sb["solves_f64"]
