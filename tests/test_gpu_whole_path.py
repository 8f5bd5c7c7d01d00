"""Whole paths of a planted dense system, the form in which the benchmark
measures paths/s: f has a planted root x* (the constant terms make f(x*) = 0
exactly); tracking x* backwards (start system f, target the total-degree
system x_i^{d_i} - 1, gamma' = 1/gamma) lands on a start root, and the forward
path of the total-degree homotopy from that root (Section 2, Eq. (1)) must end
at x*.  Checked for the corrector tolerance on every step and for the path
tolerance (tol_path) on the way: the end point against x*, against the
oracle's replay of the GPU's own schedule, and the oracle's own residual
||f(x_end)|| at the end point."""
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
@pytest.mark.parametrize("tol_path", [0.0, 1e-8])
def test_planted_whole_path(ctx, L, tol_path):
    rng = synth.Rng(606 + L)
    spec, xs = synth.planted_system(rng, 10, 10, 4, (1, 2, 3), 0.0)
    gamma = rng.unit_complex()
    params = synth.default_params(L, tol_path=tol_path, max_newton=3 if L == 2 else 5,
                                  max_steps=4000)
    f = ctx.load(spec, L)
    G = ctx.load(synth.total_degree_start(spec), L)
    gb = soa_from_complex([1.0 / gamma], L).reshape(L, 2)
    xl = np.zeros((L, 2, 10))
    st, _, _ = libph.ph_track_path(ctx.h, G, f, gb, soa_from_complex(xs, L), params, xl)
    assert st == libph.PH_OK
    x0 = soa_from_complex(synth.nearest_start_root(spec, lead_complex(xl)), L)
    gam = soa_from_complex([gamma], L).reshape(L, 2)
    xe = np.zeros_like(x0)
    st, stats, log = libph.ph_track_path(ctx.h, f, None, gam, x0, params, xe, log_cap=4001)
    assert st == libph.PH_OK and stats["t_final"] == 1.0
    # the planted root, limb by limb
    d = xe.copy()
    d[0, 0] -= xs.real
    d[0, 1] -= xs.imag
    d = d[::-1].sum(0)
    err = np.abs(d[0] + 1j * d[1]).max()
    assert err <= {2: 1e-20, 4: 1e-48}[L], err
    # the oracle's replay of the GPU's schedule ends at the same point
    of = oracle.System(spec, L)
    xr = oracle.replay(of, x0, gam, params, log)
    assert cabs_diff(xe, xr).max() <= TOL_END[L] * max(1.0, np.abs(lead_complex(xr)).max())
    # and the oracle's residual of f there is below the tolerance
    h, _ = oracle.eval_h(of, xe)
    assert np.abs(lead_complex(h)).max() < 100 * params["tol_res"]
    ctx.free(f)
    ctx.free(G)
