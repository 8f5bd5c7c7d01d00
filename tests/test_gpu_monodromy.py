"""One monodromy path on cyclic 16-roots (Section 4.2, the paper's runs of
Table 8): the solution set of dimension 3 (m = 4) cut by three random
hyperplanes L, which move to three others K, a least-squares path (N = 19
equations in n = 16 unknowns) from a start point of Backelin's family, in the
paper's form {f = 0, gamma (1-t) L + t K = 0} (the cyclic rows held fixed).

* complex double: the whole adaptive path, and the oracle's replay of its
  schedule ends at the same point (also in the form where every row moves);
* DD and QD: segments of the adaptive path replayed by the oracle (a whole
  path would take the oracle minutes), and whole paths that end on the same
  component (x_{4a+b} = i^a x_b, exact in every limb) and on the target
  slices.
"""
import numpy as np
import pytest

import oracle
from gpu_common import TOL_END, U, cabs_diff, lead_complex, soa_from_complex
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


def _mono(L, fixed=True, **over):
    """The loop in the paper's form (F = [f; K], G = [0; L], rows without a
    start term held fixed) or, fixed=False, with G = [f; L] and every row
    moving (the same zero set)."""
    F, G, gam, x0 = synth.cyclic_monodromy(1, 16, fixed=fixed)
    xs = soa_from_complex(x0, L)
    gs = soa_from_complex([gam], L).reshape(L, 2)
    return F, G, gs, xs, synth.default_params(L, fixed_rows=int(fixed), **over)


def _family_gap(x, L):
    """max |x_{4a+b} - i^a x_b| over the limbs (exact for m = 4: multiplying by
    i^a swaps or negates parts), relative to max |x|: zero on the component."""
    z = x[:, 0] + 1j * x[:, 1]                  # [L][n]
    w = np.array([1, 1j, -1, -1j])
    d = z.reshape(L, 4, 4) - w[None, :, None] * z.reshape(L, 4, 4)[:, :1, :]
    tot = d[::-1].sum(axis=0)                   # limbs summed from the smallest
    return np.abs(tot).max() / np.abs(z[0]).max()


@pytest.mark.parametrize("fixed", [True, False])
def test_monodromy_path_double_replay(ctx, fixed):
    L = 1
    F, G, gs, xs, params = _mono(L, fixed, max_steps=3000)
    f, g = ctx.load(F, L), ctx.load(G, L)
    x = np.zeros_like(xs)
    st, stats, log = libph.ph_track_path(ctx.h, f, g, gs, xs, params, x, log_cap=3100)
    assert st == libph.PH_OK and stats["t_final"] == 1.0 and len(log) == stats["steps"]
    xo = oracle.replay(oracle.System(F, L), xs, gs, params, log, g=oracle.System(G, L))
    assert cabs_diff(x, xo).max() <= TOL_END[L] * np.abs(lead_complex(xo)).max()
    assert _family_gap(x, L) < 1e-13


@pytest.mark.parametrize("L,steps,newton", [(2, 40, 5), (4, 8, 6)])
def test_monodromy_segment_replay(ctx, L, steps, newton):
    F, G, gs, xs, params = _mono(L, max_steps=steps - 1, max_newton=newton)
    f, g = ctx.load(F, L), ctx.load(G, L)
    x = np.zeros_like(xs)
    st, stats, log = libph.ph_track_path(ctx.h, f, g, gs, xs, params, x, log_cap=steps)
    assert stats["steps"] == steps and stats["accepted"] >= 1
    xo = oracle.replay(oracle.System(F, L), xs, gs, params, log, g=oracle.System(G, L))
    assert cabs_diff(x, xo).max() <= TOL_END[L]


@pytest.mark.parametrize("L,newton", [(2, 5), (4, 6)])
def test_monodromy_path_ends_on_the_component(ctx, L, newton):
    """The whole path in DD / QD: it reaches t = 1 on the same component
    (x_{4a+b} = i^a x_b to working precision) and on the target slices."""
    F, G, gs, xs, params = _mono(L, max_steps=3000, max_newton=newton)
    f, g = ctx.load(F, L), ctx.load(G, L)
    x = np.zeros_like(xs)
    st, stats, _ = libph.ph_track_path(ctx.h, f, g, gs, xs, params, x)
    assert st == libph.PH_OK and stats["t_final"] == 1.0, stats
    assert _family_gap(x, L) < 1e3 * U[L]
    h, _ = oracle.eval_h(oracle.System(F, L), x)
    assert np.abs(lead_complex(h)).max() < 1e3 * params["tol_res"]


def test_monodromy_loop_through_the_serving_loop(ctx):
    """The same loop as a serving job (one block, per-block MGS on the 19 x 16
    least-squares systems): it ends where the single-path form ends."""
    L = 2
    F, G, gs, xs, params = _mono(L, max_steps=3000, max_newton=5)
    f, g = ctx.load(F, L), ctx.load(G, L)
    x1 = np.zeros_like(xs)
    st, s1, _ = libph.ph_track_path(ctx.h, f, g, gs, xs, params, x1)
    assert st == libph.PH_OK
    srv = libph.ph_server_create(ctx.h, max_n=16, pool_bytes=1 << 26, queue_cap=4)
    try:
        jid = libph.ph_server_submit(ctx.h, srv, f, g, gs, xs, params)
        x2 = np.zeros_like(xs)
        s2, _ = libph.ph_server_wait(ctx.h, srv, jid, 60000, x2)
    finally:
        libph.ph_server_destroy(srv)
    assert s2["status"] == libph.PH_OK and s2["t_final"] == 1.0
    assert cabs_diff(x1, x2).max() <= 1e3 * params["tol_dx"]


def test_fixed_rows_needs_a_start_system(ctx):
    L = 2
    F, G, gs, xs, params = _mono(L)
    f = ctx.load(F, L)
    with pytest.raises(libph.PhError) as ei:
        libph.ph_track_path(ctx.h, f, None, gs, xs, params, np.zeros_like(xs))
    assert ei.value.status == libph.PH_EINVAL
    with pytest.raises(libph.PhError) as ei:
        libph.ph_track_paths(ctx.h, f, None, gs, np.ascontiguousarray(xs[None]), params,
                             np.zeros((1,) + xs.shape))
    assert ei.value.status == libph.PH_EINVAL


def test_fixed_rows_without_empty_rows_is_the_plain_form(ctx):
    """A start system with a term in every row: fixed_rows changes nothing, bit
    for bit, in the single-path and the many-path forms."""
    L = 2
    F, G, gs, xs, params = _mono(L, fixed=False, max_steps=29, max_newton=5)
    f, g = ctx.load(F, L), ctx.load(G, L)
    out = []
    for fr in (0, 1):
        x = np.zeros_like(xs)
        libph.ph_track_path(ctx.h, f, g, gs, xs, dict(params, fixed_rows=fr), x)
        xb = np.zeros((1,) + xs.shape)
        libph.ph_track_paths(ctx.h, f, g, gs, np.ascontiguousarray(xs[None]),
                             dict(params, fixed_rows=fr), xb)
        out.append((x, xb[0]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_monodromy_loops_find_the_degree(ctx):
    """The paper's use of these paths (Section 4.2, Table 5: degree 4 for
    n = 16): rounds of monodromy loops through the serving loop, from the
    points found so far, until a round adds nothing.  They find exactly the
    m = 4 points of the component on the start slices, each equal to one of
    the points computed from the family's linear parametrization."""
    from paper_1501_06625_gb300 import monodromy
    L, n, m = 2, 16, 4
    loop = synth.cyclic_monodromy_loop(1, n)
    params = synth.default_params(L, max_newton=5, max_steps=3000)
    res = monodromy.loops(ctx, loop, L, params, rounds=8, per_round=16, seed=3, patience=2)
    pts = [lead_complex(p) for p in res["points"]]
    assert len(pts) == m, res["found"]
    G = loop["out"][1]
    c = G.coeff.reshape(m - 1, n + 1)
    ref = monodromy.family_points_on_slices(m, c[:, :n],
                                            c[:, n] + G.coeff_lo.reshape(m - 1, n + 1)[:, n])
    for z in pts:
        assert np.abs(ref - z[None, :]).max(axis=1).min() < 1e-12


def test_monodromy_precision_form_ends_on_the_component(ctx):
    """The precision form (Newton systems in double) with the cyclic rows held
    fixed: the QD path ends on the component and on the target slices, where
    the all-QD path ends."""
    L = 4
    F, G, gs, xs, params = _mono(L, max_steps=3000, max_newton=6)
    f, g = ctx.load(F, L), ctx.load(G, L)
    x0 = np.zeros_like(xs)
    st0, _, _ = libph.ph_track_path(ctx.h, f, g, gs, xs, params, x0)
    x1 = np.zeros_like(xs)
    st1, s1, _ = libph.ph_track_path(ctx.h, f, g, gs, xs, dict(params, lin_prec=1), x1)
    assert st0 == libph.PH_OK and st1 == libph.PH_OK and s1["solves_f64"] > 0
    assert _family_gap(x1, L) < 1e3 * U[L]
    assert cabs_diff(x0, x1).max() <= 1e3 * params["tol_dx"]


def test_precision_form_leaves_an_ill_conditioned_path_to_working_precision(ctx):
    """cyclic144 in QD: the double solves of these least-squares Jacobians do
    not contract (kappa u_double near 1, far above what the pivot ratio
    shows).  The first failed low-precision corrector whose updates contracted
    only linearly sends the step, and the rest of the path, to working
    precision, which accepts steps where the double corrector accepted none."""
    L, n = 4, 144
    F, G, gam, x0 = synth.cyclic_monodromy(1, n)
    f, g = ctx.load(F, L), ctx.load(G, L)
    xs = soa_from_complex(x0, L)
    gs = soa_from_complex([gam], L).reshape(L, 2)
    params = synth.default_params(L, max_newton=6, max_steps=11, fixed_rows=1, lin_prec=1)
    x = np.zeros_like(xs)
    st, stats, log = libph.ph_track_path(ctx.h, f, g, gs, xs, params, x, log_cap=12)
    assert stats["wp_rest"] == 1 and stats["escalated"] >= 1
    assert stats["accepted"] >= 1 and stats["t_final"] > 0.0
    xo = np.zeros((1,) + xs.shape)
    sb, _ = libph.ph_track_paths(ctx.h, f, g, gs, np.ascontiguousarray(xs[None]), params, xo)
    assert (sb[0]["steps"], sb[0]["accepted"], sb[0]["wp_rest"]) == \
        (stats["steps"], stats["accepted"], 1)
