"""The continuous-batching request loop (ph_server_*): a job's result is the
same alone and in a mixed stream of double-double and quad-double jobs of
different sizes submitted while others run; served results equal the
many-path form's (whose paths the oracle checks); admission by workspace
footprint holds jobs back until pool space frees up, and every job finishes."""
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


def make_job(ctx, seed, n, prec, dense=True, steps=30):
    rng = synth.Rng(seed)
    L = 2 if prec == "dd" else 4
    spec = (synth.dense_system(rng, n, max(4, n // 2), min(4, n), (1, 2)) if dense
            else synth.sparse_system(rng, n))
    f = ctx.load(spec, L)
    g = rng.unit_complex()
    gam = soa_from_complex([g], L).reshape(L, 2)
    x0 = soa_from_complex(np.ones(n), L)
    params = synth.default_params(L, max_steps=steps - 1)
    return dict(f=f, spec=spec, gam=gam, x0=x0, params=params, L=L, n=n)


def run_alone(ctx, srv, job):
    jid = libph.ph_server_submit(ctx.h, srv, job["f"], None, job["gam"], job["x0"], job["params"])
    x = np.zeros_like(job["x0"])
    st, lat = libph.ph_server_wait(ctx.h, srv, jid, 60000, x)
    return x, st, lat


def test_same_result_alone_and_in_the_mix(ctx):
    srv = libph.ph_server_create(ctx.h, max_n=48, pool_bytes=1 << 30, queue_cap=256)
    try:
        probe = make_job(ctx, 11, 12, "dd")
        probe_qd = make_job(ctx, 12, 10, "qd")
        xa, sa, _ = run_alone(ctx, srv, probe)
        xq, sq, _ = run_alone(ctx, srv, probe_qd)
        assert sa["steps"] == 30 and sq["steps"] == 30
        mix = []
        for i in range(60):
            prec = "qd" if i % 10 < 3 else "dd"
            mix.append(make_job(ctx, 100 + i, 8 + (i * 7) % 33, prec, dense=(i % 2 == 0),
                                steps=10 + (i % 4) * 10))
        ids = []
        for i, jb in enumerate(mix):
            ids.append(libph.ph_server_submit(ctx.h, srv, jb["f"], None, jb["gam"], jb["x0"],
                                              jb["params"]))
            if i == 20:
                pa = libph.ph_server_submit(ctx.h, srv, probe["f"], None, probe["gam"],
                                            probe["x0"], probe["params"])
            if i == 40:
                pq = libph.ph_server_submit(ctx.h, srv, probe_qd["f"], None, probe_qd["gam"],
                                            probe_qd["x0"], probe_qd["params"])
        for jid, jb in zip(ids, mix):
            x = np.zeros_like(jb["x0"])
            st, lat = libph.ph_server_wait(ctx.h, srv, jid, 120000, x)
            assert st["steps"] == jb["params"]["max_steps"] + 1 or st["status"] == libph.PH_OK
        x2 = np.zeros_like(probe["x0"])
        s2, _ = libph.ph_server_wait(ctx.h, srv, pa, 60000, x2)
        x3 = np.zeros_like(probe_qd["x0"])
        s3, _ = libph.ph_server_wait(ctx.h, srv, pq, 60000, x3)
        # the tolerance of the end points; in fact the same bits
        assert cabs_diff(x2, xa).max() <= TOL_END[2] and np.array_equal(x2, xa)
        assert cabs_diff(x3, xq).max() <= TOL_END[4] and np.array_equal(x3, xq)
        assert s2 == sa and s3 == sq
    finally:
        libph.ph_server_destroy(srv)


def test_served_equals_many_path_form(ctx):
    srv = libph.ph_server_create(ctx.h, max_n=32, pool_bytes=1 << 28, queue_cap=64)
    try:
        for prec in ("dd", "qd"):
            jb = make_job(ctx, 7, 9, prec)
            xs, ss, _ = run_alone(ctx, srv, jb)
            xb = np.zeros((1,) + jb["x0"].shape)
            stats, _ = libph.ph_track_paths(ctx.h, jb["f"], None, jb["gam"],
                                            np.ascontiguousarray(jb["x0"][None]), jb["params"], xb)
            assert np.array_equal(xs, xb[0])
            assert ss["steps"] == stats[0]["steps"] and ss["newton_iters"] == stats[0]["newton_iters"]
    finally:
        libph.ph_server_destroy(srv)


def test_admission_by_footprint(ctx):
    jobs = [make_job(ctx, 300 + i, 24, "dd", steps=20) for i in range(12)]
    probe = libph.ph_server_create(ctx.h, max_n=24, pool_bytes=1 << 24, queue_cap=8)
    one = libph.ph_server_job_bytes(probe, jobs[0]["f"])
    libph.ph_server_destroy(probe)
    pool = int(2.5 * one)                     # two jobs fit at once
    srv = libph.ph_server_create(ctx.h, max_n=24, pool_bytes=pool, queue_cap=8)
    try:
        ids = [libph.ph_server_submit(ctx.h, srv, j["f"], None, j["gam"], j["x0"], j["params"])
               for j in jobs]
        info = libph.ph_server_info(srv)
        assert info["on_device"] <= 2
        assert info["waiting"] >= 8
        for jid, j in zip(ids, jobs):
            st, _ = libph.ph_server_wait(ctx.h, srv, jid, 120000, np.zeros_like(j["x0"]))
            assert st["steps"] == 20
        info = libph.ph_server_info(srv)
        assert info["waiting"] == 0 and info["on_device"] == 0
        assert info["pool_free_bytes"] == pool
    finally:
        libph.ph_server_destroy(srv)


def test_rejects_oversized_job(ctx):
    srv = libph.ph_server_create(ctx.h, max_n=8, pool_bytes=1 << 24, queue_cap=4)
    try:
        jb = make_job(ctx, 1, 12, "dd")
        with pytest.raises(libph.PhError) as ei:
            libph.ph_server_submit(ctx.h, srv, jb["f"], None, jb["gam"], jb["x0"], jb["params"])
        assert ei.value.status == libph.PH_EINVAL
    finally:
        libph.ph_server_destroy(srv)


def test_large_job_route_alone_and_in_the_mix(ctx):
    """A job above big_n (here a sparse n = 280 quad-double system, which one
    block would take minutes per solve for) runs alone on the whole GPU by the
    single-path tracker: the same bits alone and submitted in the middle of a
    stream of small jobs, which all finish; and the same end point as
    ph_track_path on the caller's context within the end-point tolerance (the
    two contexts may time their way to different solver variants)."""
    srv = libph.ph_server_create(ctx.h, max_n=32, pool_bytes=1 << 30, queue_cap=128, big_n=64)
    try:
        big = make_job(ctx, 21, 280, "qd", dense=False, steps=3)
        xa, sa, _ = run_alone(ctx, srv, big)
        assert sa["steps"] == 3 and sa["status"] in (libph.PH_OK, libph.PH_MAXSTEPS)
        mix = [make_job(ctx, 500 + i, 8 + (i * 5) % 24, "qd" if i % 4 == 0 else "dd",
                        dense=(i % 2 == 0), steps=10) for i in range(24)]
        ids = []
        for i, jb in enumerate(mix):
            ids.append(libph.ph_server_submit(ctx.h, srv, jb["f"], None, jb["gam"], jb["x0"],
                                              jb["params"]))
            if i == 11:
                pb = libph.ph_server_submit(ctx.h, srv, big["f"], None, big["gam"], big["x0"],
                                            big["params"])
        for jid, jb in zip(ids, mix):
            st, _ = libph.ph_server_wait(ctx.h, srv, jid, 300000, np.zeros_like(jb["x0"]))
            assert st["steps"] >= 1
        xb = np.zeros_like(big["x0"])
        sb, _ = libph.ph_server_wait(ctx.h, srv, pb, 300000, xb)
        assert np.array_equal(xb, xa) and sb["steps"] == sa["steps"]
        xr = np.zeros_like(big["x0"])
        libph.ph_track_path(ctx.h, big["f"], None, big["gam"], big["x0"], big["params"], xr)
        assert cabs_diff(xr, xa).max() <= TOL_END[4] * max(1.0, np.abs(lead_complex(xa)).max())
    finally:
        libph.ph_server_destroy(srv)
