"""The precision form where the Jacobian is ill-conditioned: a planted system
whose equations' coefficient moduli are 8 decades apart (rows of the Jacobian
1e8 apart in scale), tracked backwards from x* (start system f, target the
total-degree system), where the Jacobian is J_f's.  The single-path tracker in
working precision (lin_prec 0) and in the precision form (lin_prec 1: Newton
systems solved in double, residual and update in working precision) both
track the segment; the oracle replays each one's schedule in working
precision; each end point must equal its replay within the end-point
tolerance scaled by the condition number seen by the double solves, and the
two forms must end where the other's replay ends when they reach the same t."""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_END, cabs_diff, lead_complex, soa_from_complex
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


@pytest.mark.parametrize("L", [2, 4])
def test_ill_conditioned_segment_against_the_oracle(ctx, L):
    n = 16
    rng = synth.Rng(808 + L)
    spec, xs = synth.planted_system(rng, n, 16, 6, (1, 2, 3), 8.0, per_equation=True)
    gamma = rng.unit_complex()
    f = ctx.load(spec, L)
    G = ctx.load(synth.total_degree_start(spec), L)
    gb = soa_from_complex([1.0 / gamma], L).reshape(L, 2)
    x0 = soa_from_complex(xs, L)
    of, og = oracle.System(synth.total_degree_start(spec), L), oracle.System(spec, L)
    ends = {}
    for lin in (0, 1):
        params = synth.default_params(L, max_steps=19, max_dt=1e-6, max_newton=5 if L == 2 else 6,
                                      lin_prec=lin)
        xe = np.zeros_like(x0)
        st, stats, log = libph.ph_track_path(ctx.h, G, f, gb, x0, params, xe, log_cap=40)
        assert stats["accepted"] > 0
        xr = oracle.replay(of, x0, gb, params, log, g=og)
        err = cabs_diff(xe, xr).max()
        print(f"L{L} lin{lin}: {stats['accepted']} accepted, t {stats['t_final']:.3g}, "
              f"escalated {stats['escalated']}, wp_rest {stats['wp_rest']}, "
              f"cond estimate {stats['cond']:.2g}, |x - replay| {err:.2e}")
        assert err <= TOL_END[L] * max(1.0, np.abs(lead_complex(xr)).max()), err
        ends[lin] = (stats["t_final"], xe)
    if ends[0][0] == ends[1][0]:
        d = cabs_diff(ends[0][1], ends[1][1]).max()
        assert d <= 10 * TOL_END[L] * max(1.0, np.abs(lead_complex(ends[0][1])).max()), d
    ctx.free(f)
    ctx.free(G)
