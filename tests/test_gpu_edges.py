"""Edge cases of the C ABI on the GPU: an empty batch, the largest supported
exponent (and the first rejected one), the other inputs ph_system_load
rejects, and a linear target reached in one fixed step.  (The solve at
n = 1024 is checked against an exact solution in test_gpu_mgs_parity.py.)"""
import numpy as np
import pytest

import oracle
from gpu_common import assert_eval_close, lead_complex, soa_from_complex
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


def test_empty_batch_is_a_no_op(ctx):
    wl = synth.dense8(1, "dd")
    f = ctx.load(wl.f, wl.L)
    x0 = np.zeros((0, wl.L, 2, wl.n))
    stats, logs = libph.ph_track_paths(ctx.h, f, None, wl.gamma_soa(), x0, wl.params,
                                       np.zeros_like(x0))
    assert stats == [] and logs == []


@pytest.mark.parametrize("L", [1, 2, 4])
def test_largest_exponent(ctx, L):
    """Exponent 64 (the largest the power table takes) on a one-variable
    system: values and Jacobian against the oracle; 65 is rejected."""
    spec = synth.build_system(2, 2, [[(1.0, [(0, 64)]), (0.5 + 0.25j, [(1, 3)]), (-1.0, [])],
                                     [(1.0, [(0, 1), (1, 1)]), (-2.0, [])]])
    f = ctx.load(spec, L)
    x = soa_from_complex([0.99 + 0.05j, 0.7 - 0.3j], L)
    h = np.zeros((L, 2, 2))
    J = np.zeros((L, 2, 2, 2))
    tl = np.zeros(L)
    libph.ph_eval_jac(ctx.h, f, None, None, 1, tl, x, h, J)
    ho, Jo = oracle.eval_h(oracle.System(spec, L), x)
    assert_eval_close(L, spec, x, h, J, ho, Jo)
    bad = synth.build_system(1, 1, [[(1.0, [(0, 65)]), (-1.0, [])]])
    with pytest.raises(libph.PhError) as ei:
        ctx.load(bad, L)
    assert ei.value.status == libph.PH_EINVAL


@pytest.mark.parametrize("case", ["index", "repeat", "N_lt_n", "order"])
def test_system_load_rejects(ctx, case):
    spec = synth.build_system(2, 2, [[(1.0, [(0, 1)]), (1.0, [(1, 2)])], [(1.0, [(1, 1)])]])
    if case == "index":
        spec.var_idx = spec.var_idx.copy()
        spec.var_idx[0] = 5
    elif case == "repeat":
        spec = synth.build_system(2, 2, [[(1.0, [(0, 1), (0, 2)])], [(1.0, [(1, 1)])]])
    elif case == "N_lt_n":
        spec = synth.build_system(1, 2, [[(1.0, [(0, 1)]), (1.0, [(1, 1)])]])
    if case == "order":                         # term_ptr decreasing: raw arrays to the ABI
        with pytest.raises(libph.PhError) as ei:
            libph.ph_system_load(ctx.h, 2, 2, 2, np.array([0, 2, 1], dtype=np.int32),
                                 spec.var_ptr, spec.var_idx, spec.var_exp, spec.coeff_soa(2))
        assert ei.value.status == libph.PH_EINVAL
        return
    with pytest.raises(libph.PhError) as ei:
        ctx.load(spec, 2)
    assert ei.value.status == libph.PH_EINVAL


def test_linear_system_tracks_in_one_step(ctx):
    """A linear target: one fixed step from t = 0 to 1 with two updates lands
    on the solution (Newton is exact on a linear system, up to rounding)."""
    L, n = 2, 5
    rng = np.random.default_rng(4)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    spec = synth.build_system(n, n, [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])]
                                     for i in range(n)])
    f = ctx.load(spec, L)
    x0 = soa_from_complex(np.ones(n), L)
    xg = np.zeros_like(x0)
    gam = soa_from_complex([0.6 + 0.8j], L).reshape(L, 2)
    st, stats, _ = libph.ph_track_path(ctx.h, f, None, gam, x0,
                                       synth.default_params(L, fixed_steps=1, max_newton=2), xg)
    assert st == libph.PH_OK and stats["updates"] == 2
    assert np.abs(lead_complex(xg) - np.linalg.solve(A, b)).max() < 1e-12
