"""The allocation-free least-squares entry point (ph_mgs_solve_static), for
callers that cannot allocate device memory (for instance while a CUDA graph is
being captured): through the C ABI it must give the same solution as
ph_mgs_solve, within the solver tolerance of the parity tests, on two calls in
a row (the calls share one static scratch array, so the second call also
checks that the first left nothing behind that matters).  Oversized problems
are refused.  This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_common import U, cabs_diff, lead_complex, soa_from_complex, soa_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_ctx():
    from paper_1501_06625_gb300 import build, libph
    build.build()
    c = libph.Context(0)
    yield libph, c
    c.close()


@pytest.mark.parametrize("L,N,n", [(2, 64, 64), (2, 50, 33), (4, 40, 40)])
def test_static_solve_matches_context_solve(lib_ctx, L, N, n):
    libph, ctx = lib_ctx
    rng = np.random.default_rng(1234 + N + n + L)
    for call in range(2):
        A = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n))
        b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        J = soa_matrix(A, L)
        J[1] = J[0] * 2.0 ** -57
        rhs = soa_from_complex(b, L)
        dx_ref = np.zeros((L, 2, n))
        rn_ref = libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx_ref)
        dx = np.full((L, 2, n), np.nan)
        rn = libph.ph_mgs_solve_static(0, None, L, N, n, J, rhs, dx)
        kappa = np.linalg.cond(A)
        err = cabs_diff(dx, dx_ref).max() / np.abs(lead_complex(dx_ref)).max()
        assert err < 1e3 * kappa * n * U[L], (call, err)
        assert abs(rn - rn_ref) <= 1e-12 * (1 + rn_ref)


def test_static_solve_refuses_oversized(lib_ctx):
    libph, _ = lib_ctx
    n = 400
    with pytest.raises(libph.PhError) as ei:
        libph.ph_mgs_solve_static(0, None, 4, n, n, np.zeros((4, 2, n, n)), np.zeros((4, 2, n)),
                                  np.zeros((4, 2, n)))
    assert ei.value.status == libph.PH_EINVAL
