"""Parity of the least-squares solve (ph_mgs_solve: modified Gram-Schmidt on
[J | rhs] and back substitution; Introduction, and Section 2 for N >= n)
against the oracle's textbook MGS, for each solver variant pinned through
ph_mgs_set_variant, at sizes where every branch of the kernels runs:

* n = N = 288 (DD) and 260 (QD): beyond the 256 rows the grid kernel keeps in
  registers, where it also sums each pivot's norm afresh instead of
  downdating; by the grid, cluster (where it fits) and tiled kernels.  The oracle takes minutes there, so its
  solutions are stored (tests/golden/make_mgs_golden.py writes them from the
  oracle alone) and the inputs are regenerated from the seed;
* tall systems with N > 256 > n, and small square and tall shapes, by the
  grid, the cluster and the tiled kernel (one and several row blocks), in D,
  DD and QD, against the oracle live;
* n = 1024, against an exact solution: integer-valued inputs scaled by
  powers of two, whose right-hand side is computed exactly, so the solve must
  reproduce the planted dyadic solution to working precision; by the grid
  kernel and, in QD, the tiled one.

The bound is the first-order forward error of a backward-stable least-squares
solve, 2 n u (kappa + kappa^2 rho) (gpu_common.mgs_tol); each case also
reports how close it actually is, in units of n u kappa."""
import os
import sys

import numpy as np
import pytest

import oracle
from gpu_common import U, cabs_diff, complex_matrix, lead_complex, mgs_tol, soa_from_complex
from paper_1501_06625_gb300 import libph, synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_mgs_golden as golden  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1501_06625_gb300 import build
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield c
    c.close()


def _cluster_size(ctx, L, N, n):
    """The cluster size the shape takes, or 0 (probed by pinning)."""
    for C in (16, 8):
        try:
            libph.ph_mgs_set_variant(ctx.h, L, N, n, libph.MGS_CLUSTER, C)
            return C
        except libph.PhError:
            pass
    return 0


def _solve(ctx, L, N, n, J, rhs, kind, size):
    libph.ph_mgs_set_variant(ctx.h, L, N, n, kind, size)
    assert libph.ph_mgs_variant(ctx.h, L, N, n)[:2] == (kind, size if kind else 0)
    dx = np.full((L, 2, n), np.nan)
    rn = libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx)
    return dx, rn


def _compare(L, J, rhs, dx, rn, dxo, rno, label):
    A = complex_matrix(J)
    b = lead_complex(rhs)
    tol = mgs_tol(A, b, L)
    err = cabs_diff(dx, dxo).max() / np.abs(lead_complex(dxo)).max()
    kappa = np.linalg.cond(A)
    n = A.shape[1]
    print(f"{label}: |dx - oracle| / |dx| = {err:.2e}  ({err / (n * U[L] * kappa):.2e} n u kappa, "
          f"kappa {kappa:.1e}), bound {tol:.2e}")
    assert np.all(np.isfinite(dx))
    assert err <= tol, (label, err, tol)
    assert abs(rn - rno) <= 1e-12 * (1.0 + rno), (label, rn, rno)


@pytest.mark.parametrize("L,N,n", [c[:3] for c in golden.CASES])
@pytest.mark.parametrize("variant", [("grid", 0), ("cluster", 0), ("tiled", 1), ("tiled", 8)])
def test_beyond_register_cache_against_stored_oracle(ctx, L, N, n, variant):
    seed, st, rno, dxo = golden.read(L, N, n)
    assert st == oracle.OK
    J, rhs = synth.random_lsq(seed, L, N, n)
    name, size = variant
    if name == "cluster":
        size = _cluster_size(ctx, L, N, n)
        if size == 0:
            pytest.skip("the shape does not fit in a cluster's shared memory")
    kind = {"grid": libph.MGS_GRID, "cluster": libph.MGS_CLUSTER, "tiled": libph.MGS_TILED}[name]
    dx, rn = _solve(ctx, L, N, n, J, rhs, kind, size)
    _compare(L, J, rhs, dx, rn, dxo, rno, f"L{L} {N}x{n} {name} {size}")


SHAPES = [(16, 16), (64, 64), (40, 33), (300, 40), (264, 20)]
VARIANTS = [("grid", 0), ("cluster", 0), ("tiled", 1), ("tiled", 2), ("tiled", 8)]


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("N,n", SHAPES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_against_oracle(ctx, L, N, n, variant):
    if L == 4 and N == 300:
        N, n = 272, 24                                # keep the QD oracle to a second
    J, rhs = synth.random_lsq(7000 + 31 * N + n + L, L, N, n)
    name, size = variant
    if name == "cluster":
        size = _cluster_size(ctx, L, N, n)
        if size == 0:
            pytest.skip("the shape does not fit in a cluster's shared memory")
        kind = libph.MGS_CLUSTER
    else:
        kind = libph.MGS_GRID if name == "grid" else libph.MGS_TILED
    if kind == libph.MGS_TILED and N < 8 * size:
        pytest.skip("fewer than 8 rows per row block")
    dx, rn = _solve(ctx, L, N, n, J, rhs, kind, size)
    st, dxo, rno = oracle.mgs_solve(J, rhs)
    assert st == oracle.OK
    _compare(L, J, rhs, dx, rn, dxo, rno, f"L{L} {N}x{n} {name} {size}")


def test_timed_choice_is_reported(ctx):
    """Back to the timed choice: every variant that applies is timed and the
    fastest kept."""
    L, N, n = 2, 64, 64
    libph.ph_mgs_set_variant(ctx.h, L, N, n, -1)
    kind, size, ms = libph.ph_mgs_variant(ctx.h, L, N, n)
    assert ms[0] > 0 and ms[2] > 0
    applicable = [m for m in ms if m > 0]
    assert ms[kind] == min(applicable)
    print(f"DD 64x64 variant times (ms): grid {ms[0]:.3f} cluster {ms[1]:.3f} tiled {ms[2]:.3f}; "
          f"chosen {libph.MGS_KINDS[kind]} {size}")


@pytest.mark.parametrize("L", [1, 2, 4])
def test_exact_solution_at_n_1024(ctx, L):
    """A = R / 2^10 + 128 I and x* = X / 2^10 with integer R, X in [-2^10, 2^10]:
    b = A x* is computed in integers and is exact in double, so x* is the exact
    solution and the solve must reproduce it within its forward error bound
    (kappa about 2 here)."""
    n = 1024
    rng = np.random.default_rng(41 + L)
    Rr = rng.integers(-1024, 1025, (n, n))
    Ri = rng.integers(-1024, 1025, (n, n))
    Rr = Rr + 128 * 1024 * np.eye(n, dtype=np.int64)
    Xr = rng.integers(-1024, 1025, n)
    Xi = rng.integers(-1024, 1025, n)
    br = Rr @ Xr - Ri @ Xi                            # integers below 2^31: exact
    bi = Rr @ Xi + Ri @ Xr
    A = (Rr + 1j * Ri) / 1024.0
    b = (br + 1j * bi) / 2.0 ** 20
    xs = (Xr + 1j * Xi) / 1024.0
    J = np.zeros((L, 2, n, n))
    J[0, 0], J[0, 1] = A.T.real, A.T.imag
    rhs = soa_from_complex(b, L)
    dx = np.zeros((L, 2, n))
    # the grid kernel, and in QD also the tiled one
    variants = [(libph.MGS_GRID, 0)] + ([(libph.MGS_TILED, 8)] if L == 4 else [])
    for kind, size in variants:
        libph.ph_mgs_set_variant(ctx.h, L, n, n, kind, size)
        libph.ph_mgs_solve(ctx.h, L, n, n, J, rhs, dx)
        _check_exact(L, n, dx, xs, A, f"{libph.MGS_KINDS[kind]} {size}")


def _check_exact(L, n, dx, xs, A, label):
    d = dx.copy()
    d[0] -= np.stack([xs.real, xs.imag])              # exact: x* is a double
    err = np.hypot(*d.sum(0)).max() / np.abs(xs).max()
    kappa = np.linalg.cond(A)
    bound = 2 * n * U[L] * kappa
    print(f"L{L} n=1024 exact, {label}: error {err:.2e} ({err / (n * U[L] * kappa):.2e} "
          f"n u kappa), kappa {kappa:.2f}")
    assert err <= bound, (err, bound)
