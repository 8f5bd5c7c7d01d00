"""Failure detection without faulting the GPU.

* A bounded device-side wait that runs out: the least-squares solve is told to
  withhold one pivot's hand-off (ph_debug_withhold_pivot), so the blocks
  waiting for it give up after the context's wait limit (5 ms here) and the
  call returns PH_TIMEOUT; the same context then solves correctly, and a path
  whose solve times out ends with PH_TIMEOUT.
* Allocation failure on the host side: a cap on the library's device memory
  (ph_set_memory_limit) makes the next allocation fail as on a full device:
  PH_ENOMEM, with everything usable again once the cap is lifted.
* ph_server_wait on a job still running returns PH_TIMEOUT.
Nothing here faults, traps or waits beyond a bounded limit."""
import numpy as np
import pytest

import oracle
from gpu_common import cabs_diff, complex_matrix, lead_complex, mgs_tol
from paper_1501_06625_gb300 import libph, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    libph.ph_debug_withhold_pivot(c.h, -1)
    libph.ph_set_memory_limit(0)
    c.close()


@pytest.mark.parametrize("kind,size", [(libph.MGS_GRID, 0), (libph.MGS_TILED, 2)])
def test_withheld_pivot_times_out_and_the_context_recovers(ctx, kind, size):
    L, N, n = 2, 40, 40
    J, rhs = synth.random_lsq(4242, L, N, n)
    libph.ph_mgs_set_variant(ctx.h, L, N, n, kind, size)
    libph.ph_set_wait_limit(ctx.h, 5.0)
    libph.ph_debug_withhold_pivot(ctx.h, 3)
    dx = np.zeros((L, 2, n))
    try:
        with pytest.raises(libph.PhError) as ei:
            libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx)
        assert ei.value.status == libph.PH_TIMEOUT
    finally:
        libph.ph_debug_withhold_pivot(ctx.h, -1)
        libph.ph_set_wait_limit(ctx.h, 2000.0)
    libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx)
    st, dxo, _ = oracle.mgs_solve(J, rhs)
    err = cabs_diff(dx, dxo).max() / np.abs(lead_complex(dxo)).max()
    assert err <= mgs_tol(complex_matrix(J), lead_complex(rhs), L)


def test_path_whose_solve_times_out_ends_with_timeout(ctx):
    wl = synth.dense8(1, "dd")
    f = ctx.load(wl.f, wl.L)
    libph.ph_mgs_set_variant(ctx.h, wl.L, wl.n, wl.n, libph.MGS_GRID, 0)
    x0 = wl.x0_soa()
    xg = np.zeros_like(x0)
    libph.ph_set_wait_limit(ctx.h, 5.0)
    libph.ph_debug_withhold_pivot(ctx.h, 2)
    try:
        with pytest.raises(libph.PhError) as ei:
            libph.ph_track_path(ctx.h, f, None, wl.gamma_soa(), x0, wl.params, xg)
        assert ei.value.status == libph.PH_TIMEOUT
    finally:
        libph.ph_debug_withhold_pivot(ctx.h, -1)
        libph.ph_set_wait_limit(ctx.h, 2000.0)
    st, stats, _ = libph.ph_track_path(ctx.h, f, None, wl.gamma_soa(), x0, wl.params, xg)
    assert st == libph.PH_OK and stats["steps"] == 100
    ctx.free(f)


def test_memory_cap_gives_enomem_then_recovers(ctx):
    used = libph.ph_set_memory_limit(0)
    spec = synth.dense_system(synth.Rng(5), 48, 48, 8, (1, 2))
    libph.ph_set_memory_limit(used + 4096)             # too little for a new system
    try:
        with pytest.raises(libph.PhError) as ei:
            ctx.load(spec, 2)
        assert ei.value.status == libph.PH_ENOMEM
        n = 300                                         # a solve needing larger buffers
        with pytest.raises(libph.PhError) as ei:
            libph.ph_mgs_solve(ctx.h, 2, n, n, np.zeros((2, 2, n, n)), np.zeros((2, 2, n)),
                               np.zeros((2, 2, n)))
        assert ei.value.status == libph.PH_ENOMEM
    finally:
        libph.ph_set_memory_limit(0)
    f = ctx.load(spec, 2)
    assert libph.ph_set_memory_limit(0) > used
    ctx.free(f)


def test_server_wait_times_out_on_a_running_job(ctx):
    wl = synth.dense64(1, "qd")                        # seconds per path segment
    f = ctx.load(wl.f, wl.L)
    srv = libph.ph_server_create(ctx.h, max_n=64, pool_bytes=1 << 30, queue_cap=16)
    try:
        jid = libph.ph_server_submit(ctx.h, srv, f, None, wl.gamma_soa(), wl.x0_soa(),
                                     dict(wl.params, max_steps=40))
        with pytest.raises(libph.PhError) as ei:
            libph.ph_server_wait(ctx.h, srv, jid, 1)
        assert ei.value.status == libph.PH_TIMEOUT
        st, lat = libph.ph_server_wait(ctx.h, srv, jid, 600000)
        assert st["steps"] == 41 and lat > 1.0
    finally:
        libph.ph_server_destroy(srv)
    ctx.free(f)
