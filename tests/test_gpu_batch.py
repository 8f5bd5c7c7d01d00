"""GPU parity of the many-path form (ph_track_paths): every path of a batch is
checked against the oracle -- on the fixed schedule directly, on adaptive
schedules by replaying each path's own log.  Batches larger than the number
of resident blocks exercise the work queue; a non-finite start point fails
alone."""
import math

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


def start_points(spec, L, count, seed=0):
    """Total-degree start solutions x_i = exp(2 pi i m_i / d_i), rounded to
    double (the first is the all-ones root)."""
    d = spec.degrees()
    rng = np.random.default_rng(seed)
    pts = []
    for p in range(count):
        ms = np.zeros(spec.n, dtype=int) if p == 0 else rng.integers(0, d)
        z = np.exp(2j * np.pi * ms / d)
        pts.append(soa_from_complex(z, L))
    return np.ascontiguousarray(np.stack(pts))


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_batch_fixed_schedule_dense8(ctx, prec):
    wl = synth.dense8(1, prec)
    L = wl.L
    f = ctx.load(wl.f, L)
    x0 = start_points(wl.f, L, 12)
    xo = np.zeros_like(x0)
    stats, logs = libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), x0, wl.params, xo,
                                       log_cap=120)
    of = oracle.System(wl.f, L)
    for p in range(x0.shape[0]):
        assert stats[p]["status"] == libph.PH_OK
        assert stats[p]["steps"] == 100 and stats[p]["updates"] == 300
        if p % 3:                          # the oracle checks every third path
            continue
        so, xr, _, _ = oracle.track(of, x0[p], wl.gamma_soa(), wl.params)
        if not np.all(np.isfinite(xr)):
            continue
        err = cabs_diff(xo[p], xr).max()
        assert err <= TOL_END[L] * max(1.0, np.abs(lead_complex(xr)).max()), (p, err)


@pytest.mark.parametrize("L", [2, 4])
def test_batch_adaptive_replay(ctx, L):
    rng = synth.Rng(41)
    spec = synth.dense_system(rng, 5, 5, 3, (1, 2))
    g = rng.unit_complex()
    gam = soa_from_complex([g], L).reshape(L, 2)
    f = ctx.load(spec, L)
    x0 = start_points(spec, L, 6, seed=3)
    xo = np.zeros_like(x0)
    params = synth.default_params(L, max_dt=0.2, max_steps=200)
    stats, logs = libph.ph_track_paths(ctx.h, f, None, gam, x0, params, xo, log_cap=300)
    of = oracle.System(spec, L)
    for p in range(x0.shape[0]):
        assert len(logs[p]) == stats[p]["steps"]
        xr = oracle.replay(of, x0[p], gam, params, logs[p])
        err = cabs_diff(xo[p], xr).max()
        assert err <= TOL_END[L] * max(1.0, np.abs(lead_complex(xr)).max()), (p, err)


def test_batch_linear_target_converges(ctx):
    """Paths of a linear target all end at its unique solution."""
    L, n = 2, 6
    rng = np.random.default_rng(17)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    spec = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])]
                                     for i in range(n)])
    f = ctx.load(spec, L)
    x0 = np.ascontiguousarray(np.stack([soa_from_complex(np.ones(n), L)] * 3))
    xo = np.zeros_like(x0)
    gam = soa_from_complex([0.6 + 0.8j], L).reshape(L, 2)
    stats, _ = libph.ph_track_paths(ctx.h, f, None, gam, x0, synth.default_params(L), xo)
    sol = np.linalg.solve(A, b)
    for p in range(3):
        assert stats[p]["status"] == libph.PH_OK
        assert np.abs(lead_complex(xo[p]) - sol).max() < 1e-12


def test_batch_work_queue_and_nonfinite(ctx):
    """More paths than resident blocks; one path starts at NaN."""
    wl = synth.dense8(2, "dd")
    L = wl.L
    f = ctx.load(wl.f, L)
    npaths = 700
    x0 = start_points(wl.f, L, npaths, seed=5)
    x0[7, 0, 1, 2] = math.nan
    xo = np.zeros_like(x0)
    params = dict(wl.params, fixed_steps=10)
    stats, _ = libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), x0, params, xo)
    assert stats[7]["status"] == libph.PH_NONFINITE
    done = [s for i, s in enumerate(stats) if i != 7]
    assert all(s["status"] == libph.PH_OK and s["steps"] == 10 for s in done)
    # a path in the middle of the queue equals the same path tracked alone by
    # the same kernel, bit for bit (no block takes a value from another)
    alone = np.zeros_like(x0[400:401])
    libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), np.ascontiguousarray(x0[400:401]),
                         params, alone)
    assert np.array_equal(xo[400], alone[0])


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_each_summation_lane_count_matches_the_oracle(ctx, lanes):
    """The per-block summation with 1 .. 32 lanes per output (pinned): the
    fixed schedule of the dense8 system ends where the oracle's does."""
    wl = synth.dense8(1, "dd")
    L = wl.L
    f = ctx.load(wl.f, L)
    libph.ph_set_block_lanes(ctx.h, f, lanes)
    assert libph.ph_block_lanes(ctx.h, f)[0] == lanes
    x0 = start_points(wl.f, L, 2)
    xo = np.zeros_like(x0)
    stats, _ = libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), x0, wl.params, xo)
    so, xr, _, _ = oracle.track(oracle.System(wl.f, L), x0[0], wl.gamma_soa(), wl.params)
    assert stats[0]["status"] == libph.PH_OK and so == oracle.OK
    assert cabs_diff(xo[0], xr).max() <= TOL_END[L] * max(1.0, np.abs(lead_complex(xr)).max())
    ctx.free(f)


def test_summation_lanes_are_timed_on_a_full_batch(ctx):
    """A batch with at least as many paths as SMs times every lane count once
    and keeps the fastest; a smaller batch leaves the choice alone."""
    wl = synth.dense8(3, "dd")
    L = wl.L
    f = ctx.load(wl.f, L)
    params = dict(wl.params, fixed_steps=2)
    x0 = start_points(wl.f, L, 4)
    libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), x0, params, np.zeros_like(x0))
    lanes, ms = libph.ph_block_lanes(ctx.h, f)
    assert lanes == 4 and all(m == -1 for m in ms)
    x0 = start_points(wl.f, L, 304)
    libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), x0, params, np.zeros_like(x0))
    lanes, ms = libph.ph_block_lanes(ctx.h, f)
    assert all(m > 0 for m in ms)
    assert ms[[1, 2, 4, 8, 16, 32].index(lanes)] == min(ms)
    print(f"dense8 DD per-block summation: {lanes} lanes; ms by lanes {ms}")
    ctx.free(f)
