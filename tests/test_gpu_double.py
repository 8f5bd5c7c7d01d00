"""GPU parity in complex double (PH_D, one limb), the third precision of the
paper's tables: values and Jacobians against the oracle (whose one-limb
operations are IEEE double operations, pinned bit for bit against Python's
floats), the MGS solve, a fixed schedule and an adaptive path along the planted
root against the oracle, the many-path form, and the cyclic closed forms."""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_END, U, assert_eval_close, cabs_diff, lead_complex, soa_from_complex, soa_matrix
from paper_1501_06625_gb300 import libph, synth
from test_gpu_mixed import planted_case
from test_gpu_parity import CASES, _eval_both, _gamma

pytestmark = pytest.mark.gpu
L = 1


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_eval_parity_double(ctx, case):
    rng = synth.Rng(500 + len(case))
    spec = CASES[case](rng)
    x = soa_from_complex(synth.random_x(rng, spec.n), L)
    gam = _gamma(rng, L)
    h, J, ho, Jo = _eval_both(ctx, L, spec, x, 0.3713, gam, 1)
    assert_eval_close(L, spec, x, h, J, ho, Jo, t=0.3713, gamma=gam, k=1)


@pytest.mark.parametrize("N,n", [(1, 1), (8, 8), (50, 33), (64, 64)])
def test_mgs_parity_double(ctx, N, n):
    rng = np.random.default_rng(N * 1000 + n + 7)
    A = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    J, rhs = soa_matrix(A, L), soa_from_complex(b, L)
    dx = np.zeros((L, 2, n))
    libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx)
    st, dxo, _ = oracle.mgs_solve(J, rhs)
    assert st == oracle.OK
    err = cabs_diff(dx, dxo).max() / np.abs(lead_complex(dxo)).max()
    assert err < 1e3 * np.linalg.cond(A) * n * U[L], err


def test_fixed_schedule_planted_double(ctx):
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, fixed_steps=100, max_newton=3)
    xg = np.zeros_like(start)
    st, stats, _ = libph.ph_track_path(ctx.h, f, None, gam, start, params, xg)
    assert st == libph.PH_OK and stats["steps"] == 100
    _, xo, _, _ = oracle.track(of, start, gam, params)
    assert np.abs(lead_complex(xo) - xs).max() < 1e-9          # the path converges
    assert cabs_diff(xg, xo).max() <= TOL_END[L]


def test_adaptive_replay_planted_double(ctx):
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, max_steps=3000)
    xg = np.zeros_like(start)
    st, stats, log = libph.ph_track_path(ctx.h, f, None, gam, start, params, xg, log_cap=3100)
    assert st == libph.PH_OK and len(log) == stats["steps"]
    xo = oracle.replay(of, start, gam, params, log)
    assert cabs_diff(xg, xo).max() <= TOL_END[L]
    assert np.abs(lead_complex(xg) - xs).max() < 1e-9


def test_many_path_form_double(ctx):
    spec, xs, gam, start, of = planted_case(L)
    f = ctx.load(spec, L)
    params = synth.default_params(L, fixed_steps=50, max_newton=3)
    x0 = np.ascontiguousarray(np.stack([start] * 3))
    xo = np.zeros_like(x0)
    stats, _ = libph.ph_track_paths(ctx.h, f, None, gam, x0, params, xo)
    xs1 = np.zeros_like(start)
    libph.ph_track_path(ctx.h, f, None, gam, start, params, xs1)
    for p in range(3):
        assert stats[p]["status"] == libph.PH_OK and stats[p]["steps"] == 50
        assert cabs_diff(xo[p], xs1).max() <= TOL_END[L]


def test_cyclic_closed_form_double(ctx):
    n = 128
    f = ctx.load(synth.cyclic_system(n), L)
    x = soa_from_complex(np.ones(n), L)
    h = np.zeros((L, 2, n))
    J = np.zeros((L, 2, n, n))
    tl = np.zeros(L)
    libph.ph_eval_jac(ctx.h, f, None, None, 1, tl, x, h, J)
    want_h = np.full(n, float(n))
    want_h[-1] = 0.0
    assert np.array_equal(h[0, 0], want_h) and not np.any(h[0, 1])
    want_J = np.tile(np.arange(1, n + 1, dtype=float), (n, 1))
    want_J[:, -1] = 1.0
    assert np.array_equal(J[0, 0], want_J) and not np.any(J[0, 1])
