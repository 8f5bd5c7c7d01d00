"""Pins of the oracle's predictor, Newton corrector and step-size control.

* Step control: scripted success/failure sequences against traces derived by
  hand from the path-tracking pseudocode (Fig. 3) with the readings in the oracle's header.
* Predictor: the extrapolation reproduces any polynomial of degree <= p
  through p+1 points, and for degree p+1 data misses by exactly the
  interpolation remainder c_{p+1} prod (t - t_j) (mpmath).
* Homotopies with known paths:
  - f = g: the path stays on the start root exactly;
  - linear f = A x - b: Newton on a linear system is exact, so every accepted
    point and the end point solve a known linear system (mpmath);
  - n = 1, f = x^3 - c: x(t)^3 = (gamma (1-t) + t c) / (gamma (1-t) + t).
* Replay of an adaptive run's own schedule reproduces its end point bit for bit.
"""
import numpy as np
import pytest

from paper_1501_06625_gb300 import synth
from refmath import mp_vec, soa_from_complex

mpmath = pytest.importorskip("mpmath")


def _params(**kw):
    p = synth.default_params(2)
    p.update(kw)
    return p


def _drive(orc, params, outcomes):
    c = orc.Controller(params)
    ts = []
    for ok in outcomes:
        t = c.next_t()
        if t < 0:
            break
        ts.append(t)
        c.report(t, ok)
    return ts, c


def test_controller_trace(orc):
    ts, c = _drive(orc, _params(max_dt=0.25, min_dt=0.01),
                   [1, 0, 1, 1, 1, 1, 0, 1, 1])
    assert ts == [0.25, 0.5, 0.375, 0.5, 0.625, 0.875, 1.0, 1.0]
    st = c.state
    assert st["done"] == 1 and st["status"] == orc.OK and st["t"] == 1.0
    assert st["nsteps"] == 8


def test_controller_doubling_rule(orc):
    # dt doubles on the third success in a row and on each one after (capped)
    ts, c = _drive(orc, _params(max_dt=0.25, min_dt=0.01), [0, 0, 1, 1, 1, 1, 1])
    # failures: dt 0.25 -> 0.125 -> 0.0625; then t = 0.0625, 0.125, 0.1875 (third
    # success doubles to 0.125), 0.3125 (doubles to 0.25), 0.5625
    assert ts == [0.25, 0.125, 0.0625, 0.125, 0.1875, 0.3125, 0.5625]
    assert c.state["dt"] == 0.25


def test_controller_stepmin_and_maxsteps(orc):
    ts, c = _drive(orc, _params(max_dt=0.25, min_dt=0.1), [0, 0, 0])
    assert ts == [0.25, 0.125] and c.state["status"] == orc.STEPMIN
    ts, c = _drive(orc, _params(max_dt=0.25, min_dt=1e-9, max_steps=2), [0] * 10)
    assert len(ts) == 3 and c.state["status"] == orc.MAXSTEPS


def test_controller_fixed_schedule(orc):
    ts, c = _drive(orc, _params(fixed_steps=4), [0, 1, 0, 1, 1])
    assert ts == [0.25, 0.5, 0.75, 1.0] and c.state["done"] == 1


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("p", [0, 1, 2, 4])
def test_predictor_polynomial_data(orc, L, p):
    mp = mpmath.mp
    mp.prec = 400
    rng = np.random.default_rng(p + 10 * L)
    n = 3
    ts = np.array([0.0, 0.1, 0.25, 0.3, 0.45, 0.5][: p + 2])
    coefs = rng.standard_normal((p + 2, n)) + 1j * rng.standard_normal((p + 2, n))

    def poly(deg, t):
        return [sum(mp.mpc(coefs[e, i].real, coefs[e, i].imag) * mp.mpf(t) ** e
                    for e in range(deg + 1)) for i in range(n)]

    tn = 0.6
    u = 2.0 ** (-53 * L)
    from refmath import soa_from_mp
    for deg in (p, p + 1):
        xs = np.stack([soa_from_mp(poly(deg, t), L, mp) for t in ts[: p + 1]])
        got = mp_vec(orc.predict(ts[: p + 1], xs, tn), mp)
        want = poly(deg, tn)
        if deg == p + 1:                       # interpolation remainder
            rem = mp.mpf(1)
            for t in ts[: p + 1]:
                rem *= mp.mpf(tn) - mp.mpf(t)
            want = [want[i] - mp.mpc(coefs[deg, i].real, coefs[deg, i].imag) * rem
                    for i in range(n)]
        for i in range(n):
            assert abs(got[i] - want[i]) < 1e4 * u * (1 + abs(want[i]))


def test_f_equals_g_stays_on_root(orc):
    L, n = 2, 4
    spec = synth.build_system(n, n, [[(1.0, [(i, 3)]), (-1.0, [])] for i in range(n)])
    f = orc.System(spec, L)
    gam = np.zeros((L, 2)); gam[0] = [0.6, 0.8]
    x0 = soa_from_complex(np.ones(n), L)
    status, x, st, log = orc.track(f, x0, gam, _params())
    assert status == orc.OK and st["t_final"] == 1.0
    assert np.array_equal(x, x0)
    assert all(r["accepted"] and r["updates"] == 0 for r in log)


def _linear_system(rng, n):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    polys = [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])] for i in range(n)]
    return A, b, synth.build_system(n, n, polys)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("fixed", [0, 8])
def test_linear_target(orc, L, fixed):
    mp = mpmath.mp
    mp.prec = 400
    rng = np.random.default_rng(17)
    n = 4
    A, b, spec = _linear_system(rng, n)
    f = orc.System(spec, L)
    gam = np.zeros((L, 2)); gam[0] = [0.6, 0.8]
    x0 = soa_from_complex(np.ones(n), L)
    status, x, st, log = orc.track(f, x0, gam, _params(fixed_steps=fixed, max_newton=2) if fixed
                                   else synth.default_params(L))
    assert status == orc.OK
    Am = mp.matrix([[mp.mpc(A[i, j].real, A[i, j].imag) for j in range(n)] for i in range(n)])
    bm = mp.matrix([mp.mpc(v.real, v.imag) for v in b])
    xs = mp.lu_solve(Am, bm)
    got = mp_vec(x, mp)
    u = 2.0 ** (-53 * L)
    assert max(abs(got[i] - xs[i]) for i in range(n)) < 1e3 * u * np.linalg.cond(A)


@pytest.mark.parametrize("L", [2, 4])
def test_one_variable_closed_form(orc, L):
    mp = mpmath.mp
    mp.prec = 400
    c = 0.3 + 0.4j
    spec = synth.build_system(1, 1, [[(1.0, [(0, 3)]), (-c, [])]])
    f = orc.System(spec, L)
    g = complex(np.cos(1.1), np.sin(1.1))
    gam = np.zeros((L, 2)); gam[0] = [g.real, g.imag]
    x0 = soa_from_complex([1.0], L)
    u = 2.0 ** (-53 * L)
    params = synth.default_params(L)
    status, x, st, log = orc.track(f, x0, gam, params)
    assert status == orc.OK
    cm = mp.mpc(c.real, c.imag)
    # the corrector stops once the residual or the update is below tolerance
    assert abs(mp_vec(x, mp)[0] ** 3 - cm) < 10 * max(params["tol_res"], params["tol_dx"])
    # two more Newton steps at t = 1 reach working precision
    _, xr, _, _, _, _ = orc.newton(f, x, 1.0, gam, dict(params, max_newton=2), fixed=True)
    assert abs(mp_vec(xr, mp)[0] ** 3 - cm) < 100 * u
    # the corrector at an interior t converges to the closed-form point
    t = 0.5
    gm = mp.mpc(g.real, g.imag)
    w = ((gm * (1 - t) + t * cm) / (gm * (1 - t) + t)) ** (mp.mpf(1) / 3)
    from refmath import soa_from_mp
    start = soa_from_mp([w * (1 + mp.mpf("1e-6"))], L, mp)
    ok, xn, iters, upd, res, dxn = orc.newton(f, start, t, gam, synth.default_params(L, max_newton=8))
    assert ok
    assert abs(mp_vec(xn, mp)[0] - w) < 100 * u


def test_replay_reproduces_adaptive_run(orc):
    L = 2
    rng = synth.Rng(4)
    spec = synth.dense_system(rng, 3, 3, 2, (1, 2))
    f = orc.System(spec, L)
    gam = np.zeros((L, 2)); g = rng.unit_complex(); gam[0] = [g.real, g.imag]
    x0 = soa_from_complex(np.ones(3), L)
    params = synth.default_params(L, max_dt=0.5)
    status, x, st, log = orc.track(f, x0, gam, params)
    assert st["steps"] == len(log) > 3
    xr = orc.replay(f, x0, gam, params, log)
    assert np.array_equal(xr, x)


def test_nonfinite_start(orc):
    L = 2
    spec = synth.build_system(2, 2, [[(1.0, [(0, 2)]), (-1.0, [])], [(1.0, [(1, 2)]), (-1.0, [])]])
    f = orc.System(spec, L)
    gam = np.zeros((L, 2)); gam[0] = [0.6, 0.8]
    x0 = soa_from_complex([1.0, np.nan], L)
    status, x, st, log = orc.track(f, x0, gam, synth.default_params(L))
    assert status == orc.NONFINITE and not log


@pytest.mark.parametrize("L", [2, 4])
def test_path_tolerance_applies_before_t_1_only(orc, L):
    """With tol_path > 0 the corrector's tests use it on the steps to t < 1,
    and tol_res / tol_dx on the step that lands on t = 1: the interior steps
    stop as soon as an update is below tol_path (some well above tol_dx, so the
    path takes fewer corrector iterations), while the end point still meets
    the closed form x(1)^3 = c to the working-precision tolerance."""
    mp = mpmath.mp
    mp.prec = 400
    c = 0.3 + 0.4j
    spec = synth.build_system(1, 1, [[(1.0, [(0, 3)]), (-c, [])]])
    f = orc.System(spec, L)
    g = complex(np.cos(1.1), np.sin(1.1))
    gam = np.zeros((L, 2)); gam[0] = [g.real, g.imag]
    x0 = soa_from_complex([1.0], L)
    tight = synth.default_params(L)
    loose = dict(tight, tol_path=1e-6)
    st0, x_t, s_t, log_t = orc.track(f, x0, gam, tight)
    st1, x_l, s_l, log_l = orc.track(f, x0, gam, loose)
    assert st0 == orc.OK and st1 == orc.OK
    interior = [r for r in log_l if r["accepted"] and r["t"] < 1.0]
    assert interior and all(min(r["res"], r["dx"]) < 1e-6 for r in interior)
    assert any(r["dx"] > tight["tol_dx"] and r["res"] > tight["tol_res"] for r in interior)
    last = log_l[-1]
    assert last["t"] == 1.0 and last["accepted"]
    assert min(last["res"], last["dx"]) < tight["tol_res"]
    assert s_l["newton_iters"] < s_t["newton_iters"]
    cm = mp.mpc(c.real, c.imag)
    assert abs(mp_vec(x_l, mp)[0] ** 3 - cm) < 10 * tight["tol_res"]
