"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.

* ph_eval_jac: values and Jacobians of the homotopy, every element, within
  1e-28 (DD) / 1e-58 (QD) of the oracle relative to the sum of the term
  magnitudes; cases span several warps and a ragged tail, constants, deep
  exponents, k = 2, a general start system, f alone, and the full-size dense
  n = 64 (4096 monomials over 16 variables) and sparse n = 512 systems.
* ph_mgs_solve: solutions of square and tall systems against the oracle's
  textbook MGS within the first-order least-squares forward error bound
  2 n u (kappa + kappa^2 rho); rank deficiency is reported.
* ph_track_path: the fixed schedule of the 8-variable dense system (100 steps,
  3 updates each) ends within 1e-24 (DD) / 1e-52 (QD) of the oracle; adaptive
  runs are replayed by the oracle from the GPU's own step log and must end at
  the same tolerance.
"""
import numpy as np
import pytest

import oracle
from gpu_common import (TOL_END, assert_eval_close, cabs_diff, complex_matrix, lead_complex,
                        mgs_tol, soa_from_complex, soa_matrix)
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


def _gamma(rng, L):
    g = rng.unit_complex()
    return soa_from_complex([g], L).reshape(L, 2)


def _ragged_system(rng, n):
    """Terms with 0..6 distinct variables, exponents up to 7, a constant in
    every polynomial, and a term count that is not a multiple of 32."""
    polys = []
    for i in range(n):
        terms = [(rng.unit_complex(), [])]
        for _ in range(3 + (i % 5)):
            v = 1 + rng.below(6)
            vs = rng.sample(n, v)
            terms.append((rng.unit_complex(), [(u, 1 + rng.below(7)) for u in vs]))
        terms.append((rng.unit_complex(), [(i, 1 + rng.below(3))]))
        polys.append(terms)
    return synth.build_system(n, n, polys)


CASES = {
    "dense8": lambda r: synth.dense_system(r, 8, 8, 4, (1, 2)),
    "dense20": lambda r: synth.dense_system(r, 20, 24, 5, (1, 2, 3, 4)),
    "ragged13": lambda r: _ragged_system(r, 13),
    "sparse40": lambda r: synth.sparse_system(r, 40),
}


def _eval_both(ctx, L, spec, x, t, gam, k, gspec=None):
    f = ctx.load(spec, L)
    g = ctx.load(gspec, L) if gspec is not None else None
    n, N = spec.n, spec.N
    h = np.zeros((L, 2, N))
    J = np.zeros((L, 2, n, N))
    tl = np.zeros(L); tl[0] = t
    libph.ph_eval_jac(ctx.h, f, g, gam, k, tl, x, h, J)
    of = oracle.System(spec, L)
    og = oracle.System(gspec, L) if gspec is not None else None
    ho, Jo = oracle.eval_h(of, x, t=t, gamma=gam, k=k, g=og)
    return h, J, ho, Jo


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("mode", ["homotopy_k1", "homotopy_k2", "f_only"])
def test_eval_parity(ctx, L, case, mode):
    rng = synth.Rng(100 + len(case) + 7 * L)
    spec = CASES[case](rng)
    x = soa_from_complex(synth.random_x(rng, spec.n), L)
    x[1] = x[0] * 2.0 ** -55                         # use the low limb too
    gam = _gamma(rng, L)
    if mode == "f_only":
        h, J, ho, Jo = _eval_both(ctx, L, spec, x, 0.0, None, 1)
        assert_eval_close(L, spec, x, h, J, ho, Jo)
    else:
        k = 1 if mode.endswith("k1") else 2
        t = 0.3713
        h, J, ho, Jo = _eval_both(ctx, L, spec, x, t, gam, k)
        assert_eval_close(L, spec, x, h, J, ho, Jo, t=t, gamma=gam, k=k)


@pytest.mark.parametrize("L", [2, 4])
def test_eval_general_start_system(ctx, L):
    rng = synth.Rng(77)
    spec = synth.dense_system(rng, 9, 7, 3, (1, 2, 3))
    gspec = synth.dense_system(rng, 9, 5, 2, (1, 2))
    x = soa_from_complex(synth.random_x(rng, 9), L)
    gam = _gamma(rng, L)
    h, J, ho, Jo = _eval_both(ctx, L, spec, x, 0.61, gam, 1, gspec)
    assert_eval_close(L, spec, x, h, J, ho, Jo, t=0.61, gamma=gam, k=1, g=gspec)


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_eval_full_size_dense64(ctx, prec):
    wl = synth.dense64(1, prec)
    L = wl.L
    rng = synth.Rng(5)
    x = soa_from_complex(synth.random_x(rng, wl.n), L)
    h, J, ho, Jo = _eval_both(ctx, L, wl.f, x, 0.25, wl.gamma_soa(), 1)
    assert_eval_close(L, wl.f, x, h, J, ho, Jo, t=0.25, gamma=wl.gamma_soa(), k=1)


def test_eval_full_size_sparse512(ctx):
    wl = synth.sparse512(1, "qd")
    L = wl.L
    rng = synth.Rng(6)
    x = soa_from_complex(synth.random_x(rng, wl.n), L)
    h, J, ho, Jo = _eval_both(ctx, L, wl.f, x, 0.8, wl.gamma_soa(), 1)
    assert_eval_close(L, wl.f, x, h, J, ho, Jo, t=0.8, gamma=wl.gamma_soa(), k=1)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("N,n", [(1, 1), (8, 8), (37, 37), (50, 33), (64, 64)])
def test_mgs_parity(ctx, L, N, n):
    """The solve of whichever variant the context picks by timing (each variant
    pinned, and the sizes beyond 256 rows: test_gpu_mgs_parity.py)."""
    rng = np.random.default_rng(N * 1000 + n + L)
    A = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    J = soa_matrix(A, L)
    J[1] = J[0] * 2.0 ** -60
    rhs = soa_from_complex(b, L)
    dx = np.zeros((L, 2, n))
    rn = libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx)
    st, dxo, rno = oracle.mgs_solve(J, rhs)
    assert st == oracle.OK
    err = cabs_diff(dx, dxo).max() / np.abs(lead_complex(dxo)).max()
    assert err <= mgs_tol(complex_matrix(J), lead_complex(rhs), L), err
    assert abs(rn - rno) <= 1e-12 * (1 + rno)


def test_mgs_rank_deficient(ctx):
    A = np.eye(5, dtype=complex)
    A[:, 3] = A[:, 1]
    with pytest.raises(libph.PhError) as ei:
        libph.ph_mgs_solve(ctx.h, 2, 5, 5, soa_matrix(A, 2), soa_from_complex(np.ones(5), 2),
                           np.zeros((2, 2, 5)))
    assert ei.value.status == libph.PH_NONFINITE


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_track_fixed_schedule_dense8(ctx, prec):
    """The 8-variable dense system, 100 fixed steps with exactly 3 updates."""
    wl = synth.dense8(1, prec)
    L = wl.L
    f = ctx.load(wl.f, L)
    x0, gam = wl.x0_soa(), wl.gamma_soa()
    xg = np.zeros_like(x0)
    st, stats, log = libph.ph_track_path(ctx.h, f, None, gam, x0, wl.params, xg, log_cap=200)
    assert st == libph.PH_OK
    assert stats["steps"] == 100 and stats["updates"] == 300 and len(log) == 100
    so, xo, ostats, _ = oracle.track(oracle.System(wl.f, L), x0, gam, wl.params)
    assert so == oracle.OK
    assert np.all(np.isfinite(xg))
    err = cabs_diff(xg, xo).max()
    assert err <= TOL_END[L], err


def _replay_check(ctx, spec, L, gam, x0, params, log_cap=5000):
    f = ctx.load(spec, L)
    xg = np.zeros_like(x0)
    st, stats, log = libph.ph_track_path(ctx.h, f, None, gam, x0, params, xg, log_cap=log_cap)
    assert len(log) == stats["steps"] <= log_cap, "the schedule log must hold the whole path"
    xo = oracle.replay(oracle.System(spec, L), x0, gam, params, log)
    err = cabs_diff(xg, xo).max()
    assert err <= TOL_END[L] * max(1.0, np.abs(lead_complex(xo)).max()), err
    return st, stats, log


@pytest.mark.parametrize("L", [2, 4])
def test_track_linear_target_replay(ctx, L):
    """A linear target (paths converge): the whole adaptive path, replayed."""
    rng = np.random.default_rng(17)
    n = 6
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    spec = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])]
                                     for i in range(n)])
    gam = soa_from_complex([0.6 + 0.8j], L).reshape(L, 2)
    st, stats, log = _replay_check(ctx, spec, L, gam, soa_from_complex(np.ones(n), L),
                                   synth.default_params(L))
    assert st == libph.PH_OK


@pytest.mark.parametrize("L", [2, 4])
def test_track_adaptive_replay(ctx, L):
    rng = synth.Rng(31)
    spec = synth.dense_system(rng, 5, 5, 3, (1, 2))
    gam = _gamma(rng, L)
    x0 = soa_from_complex(np.ones(5), L)
    # this path is hard (both sides reach t ~ 0.6 in 300 steps): compare the
    # first 301 steps, rejections included
    st, stats, log = _replay_check(ctx, spec, L, gam, x0,
                                   synth.default_params(L, max_dt=0.2, max_steps=300))
    assert stats["steps"] == 301 and stats["rejected"] > 0


def test_track_dense64_replay_first_steps(ctx):
    """The bench's workload in DD at full size: the first 6 steps of the
    adaptive path, replayed by the oracle."""
    wl = synth.dense64(1, "dd")
    params = dict(wl.params, max_steps=5)
    st, stats, log = _replay_check(ctx, wl.f, 2, wl.gamma_soa(), wl.x0_soa(), params)
    assert st in (libph.PH_OK, libph.PH_MAXSTEPS)
    assert stats["steps"] == 6


@pytest.mark.parametrize("L", [2, 4])
def test_host_control_matches_device_loop(ctx, L):
    """The paper's host-side step control (one launch per step, the state read
    back after each) runs the same kernels: the same log and end point."""
    rng = synth.Rng(31)
    spec = synth.dense_system(rng, 5, 5, 3, (1, 2))
    gam = _gamma(rng, L)
    x0 = soa_from_complex(np.ones(5), L)
    f = ctx.load(spec, L)
    out = []
    for control in (0, 1):
        p = synth.default_params(L, max_dt=0.2, max_steps=60, control=control)
        xg = np.zeros_like(x0)
        st, stats, log = libph.ph_track_path(ctx.h, f, None, gam, x0, p, xg, log_cap=100)
        out.append((st, stats, log, xg))
    assert out[0][0] == out[1][0]
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][3], out[1][3])
    assert out[1][1]["launches"] == out[0][1]["launches"]


def test_track_f_equals_g(ctx):
    n, L = 4, 2
    spec = synth.build_system(n, n, [[(1.0, [(i, 3)]), (-1.0, [])] for i in range(n)])
    f = ctx.load(spec, L)
    x0 = soa_from_complex(np.ones(n), L)
    xg = np.zeros_like(x0)
    gam = soa_from_complex([0.6 + 0.8j], L).reshape(L, 2)
    st, stats, log = libph.ph_track_path(ctx.h, f, None, gam, x0, synth.default_params(L), xg,
                                         log_cap=100)
    assert st == libph.PH_OK and stats["t_final"] == 1.0
    # the extrapolation of identical points rounds its weights' sum: within tolerance of 1
    assert cabs_diff(xg, x0).max() <= TOL_END[L]


def test_track_nonfinite_start(ctx):
    wl = synth.dense8(1, "dd")
    f = ctx.load(wl.f, 2)
    x0 = wl.x0_soa()
    x0[0, 1, 3] = np.nan
    xg = np.zeros_like(x0)
    st, stats, log = libph.ph_track_path(ctx.h, f, None, wl.gamma_soa(), x0, wl.params, xg)
    assert st == libph.PH_NONFINITE


def test_invalid_arguments(ctx):
    bad = synth.build_system(2, 2, [[(1.0, [(0, 1), (0, 2)])], [(1.0, [(1, 1)])]])
    with pytest.raises(libph.PhError) as ei:
        ctx.load(bad, 2)
    assert ei.value.status == libph.PH_EINVAL
    with pytest.raises(libph.PhError):
        libph.ph_mgs_solve(ctx.h, 2, 3, 5, np.zeros((2, 2, 5, 3)), np.zeros((2, 2, 3)),
                           np.zeros((2, 2, 5)))


def _first_decision_difference(glog, olog):
    """Index of the first step whose (t, accepted, updates) differ, or None."""
    for i, (a, b) in enumerate(zip(glog, olog)):
        if a["t"] != b["t"] or a["accepted"] != b["accepted"] or a["updates"] != b["updates"]:
            return i
    return None if len(glog) == len(olog) else min(len(glog), len(olog))


def _near_threshold(rec, params, rel=1e-6):
    """A corrector outcome decided by a norm within rounding of its tolerance."""
    return any(abs(rec[k] / params[tk] - 1.0) < rel
               for k, tk in (("res", "tol_res"), ("dx", "tol_dx")) if rec[k] > 0)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("case", ["linear6", "dense5_first300", "dense64_first10"])
def test_step_decisions_against_the_oracle(ctx, L, case):
    """The library and the oracle each track the path and take their own
    decisions (Fig. 3 step control, Fig. 2 corrector tests); their schedules
    (every t tried, accepted or not, updates applied) must be identical until a
    decision that rests on a norm within rounding of its tolerance, and the
    end points must then agree to the end-point tolerance."""
    if case == "linear6":
        rng = np.random.default_rng(17)
        n = 6
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        spec = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])]
                                         for i in range(n)])
        gam = soa_from_complex([0.6 + 0.8j], L).reshape(L, 2)
        x0 = soa_from_complex(np.ones(n), L)
        params = synth.default_params(L)
    elif case == "dense5_first300":
        rng = synth.Rng(31)
        spec = synth.dense_system(rng, 5, 5, 3, (1, 2))
        gam = _gamma(rng, L)
        x0 = soa_from_complex(np.ones(5), L)
        params = synth.default_params(L, max_dt=0.2, max_steps=299)
    else:
        if L == 4:
            pytest.skip("the QD dense64 oracle steps take minutes; DD covers the full size")
        wl = synth.dense64(1, "dd")
        spec, gam, x0 = wl.f, wl.gamma_soa(), wl.x0_soa()
        params = dict(wl.params, max_steps=9)
    f = ctx.load(spec, L)
    xg = np.zeros_like(x0)
    st, stats, glog = libph.ph_track_path(ctx.h, f, None, gam, x0, params, xg, log_cap=20000)
    so, xo, ostats, olog = oracle.track(oracle.System(spec, L), x0, gam, params)
    i = _first_decision_difference(glog, olog)
    print(f"{case} L{L}: {len(glog)} steps, first differing decision: {i}")
    if i is not None:
        assert _near_threshold(glog[i], params) or _near_threshold(olog[i], params), (i, glog[i],
                                                                                      olog[i])
        return
    assert st == so and stats["steps"] == ostats["steps"]
    assert stats["accepted"] == ostats["accepted"] and stats["updates"] == ostats["updates"]
    err = cabs_diff(xg, xo).max()
    assert err <= TOL_END[L] * max(1.0, np.abs(lead_complex(xo)).max()), err


def test_track_after_a_system_is_freed_and_another_loaded(ctx):
    """A path graph is cached per context; freeing a system and loading
    another of the same shape (which may get the freed one's address) must not
    replay the old graph.  The second system is linear, so its fixed schedule
    (Newton exact on a linear system) ends on the solution A^-1 b."""
    L, n = 2, 8
    wl = synth.dense8(1, "dd")
    params = wl.params
    f = ctx.load(wl.f, L)
    xg = np.zeros_like(wl.x0_soa())
    st, _, _ = libph.ph_track_path(ctx.h, f, None, wl.gamma_soa(), wl.x0_soa(), params, xg)
    ctx.free(f)
    assert st == libph.PH_OK
    rng = np.random.default_rng(88)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    spec = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])]
                                     for i in range(n)])
    f2 = ctx.load(spec, L)
    x0 = soa_from_complex(np.ones(n), L)
    xg = np.zeros_like(x0)
    st, _, _ = libph.ph_track_path(ctx.h, f2, None, wl.gamma_soa(), x0, params, xg)
    ctx.free(f2)
    assert st == libph.PH_OK
    so, xo, _, _ = oracle.track(oracle.System(spec, L), x0, wl.gamma_soa(), params)
    assert so == oracle.OK
    assert np.abs(lead_complex(xg) - np.linalg.solve(A, b)).max() < 1e-12
    assert cabs_diff(xg, xo).max() <= TOL_END[L]
