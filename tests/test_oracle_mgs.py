"""Pins of the oracle's modified Gram-Schmidt least-squares solver.

* Q^H Q = I and Q R = [J | rhs] to working precision, checked in 400-bit
  mpmath for square and tall (N > n, least squares) systems.
* The solution against the exact least-squares solution (mpmath), within
  kappa * u; for N > n the normal equations J^H (J dx - rhs) = 0 hold.
* Upper-triangular J with unit-phase diagonal and dyadic entries: MGS must
  return Q = diag(phase), R = diag(conj phase) J exactly and the exact
  solution of the triangular system (fractions).
* Agreement with numpy's double-precision least squares (a library special
  case) to double accuracy.
* A zero column makes r_kk = 0: the solver reports NONFINITE.
"""
from fractions import Fraction

import numpy as np
import pytest

from refmath import frac_vec, mp_vec, soa_from_complex

mpmath = pytest.importorskip("mpmath")


def _rand_complex(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _soa_mat(A, L):
    """complex N x n -> [L][2][n][N] column-major."""
    N, n = A.shape
    out = np.zeros((L, 2, n, N))
    out[0, 0] = A.T.real
    out[0, 1] = A.T.imag
    return out


def _mp_mat(M, mp):
    """[L][2][cols][rows] -> mpmath matrix rows x cols."""
    L, _, c, r = M.shape
    out = mp.matrix(r, c)
    for j in range(c):
        col = mp_vec(M[:, :, j, :], mp)
        for i in range(r):
            out[i, j] = col[i]
    return out


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("N,n", [(6, 6), (9, 5), (12, 12)])
def test_qr_properties(orc, L, N, n):
    mp = mpmath.mp
    mp.prec = 400
    rng = np.random.default_rng(N * 10 + n + L)
    A = _rand_complex(rng, (N, n))
    b = _rand_complex(rng, N)
    J, rhs = _soa_mat(A, L), soa_from_complex(b, L)
    st, dx, rn, Q, R = orc.mgs_solve(J, rhs, want_qr=True)
    assert st == orc.OK
    u = 2.0 ** (-53 * L)
    Qm = _mp_mat(Q, mp)
    Rm = _mp_mat(R, mp)                       # (n+1) x (n+1)
    QhQ = Qm.H * Qm
    assert max(abs(QhQ[i, j] - (1 if i == j else 0)) for i in range(n) for j in range(n)) < 10 * n * u
    # Q R[:n, :] reproduces [J | rhs] (the last column up to the residual vector)
    Jm = _mp_mat(J, mp)
    bm = mp_vec(rhs, mp)
    QR = Qm * Rm[0:n, 0:n + 1]
    nrm = max(abs(Jm[i, j]) for i in range(N) for j in range(n))
    assert max(abs(QR[i, j] - Jm[i, j]) for i in range(N) for j in range(n)) < 10 * n * u * nrm
    # R is upper triangular with a real positive diagonal
    for j in range(n + 1):
        assert Rm[j, j].imag == 0 and Rm[j, j].real >= 0
        for i in range(j + 1, n + 1):
            assert Rm[i, j] == 0
    # exact least-squares solution and normal equations
    xs = mp.qr_solve(Jm, mp.matrix(bm))[0] if N > n else mp.lu_solve(Jm, mp.matrix(bm))
    dxm = mp_vec(dx, mp)
    cond = np.linalg.cond(A)
    err = max(abs(dxm[i] - xs[i]) for i in range(n)) / max(abs(xs[i]) for i in range(n))
    assert err < 50 * n * cond * u
    r = Jm * mp.matrix(dxm) - mp.matrix(bm)
    ne = Jm.H * r
    assert max(abs(ne[i]) for i in range(n)) < 50 * n * cond * u * nrm * nrm * max(abs(v) for v in xs)
    # the reported residual norm is ||J dx - rhs||_2
    assert abs(rn - float(mp.norm(r))) <= 1e-12 * (1 + abs(rn)) + 100 * n * u * float(mp.norm(mp.matrix(bm)))


@pytest.mark.parametrize("L", [2, 4])
def test_triangular_exact(orc, L):
    n = 5
    rng = np.random.default_rng(4)
    phases = np.array([1, 1j, -1, -1j, 1j])
    A = np.triu((rng.integers(-8, 9, (n, n)) + 1j * rng.integers(-8, 9, (n, n))) / 8.0, 1)
    A += np.diag(phases)
    b = (rng.integers(-8, 9, n) + 1j * rng.integers(-8, 9, n)) / 4.0
    st, dx, rn, Q, R = orc.mgs_solve(_soa_mat(A, L), soa_from_complex(b, L), want_qr=True)
    assert st == orc.OK
    # Q = diag(phases) exactly
    for j in range(n):
        col = frac_vec(Q[:, :, j, :])
        for i in range(n):
            want = (Fraction(phases[j].real), Fraction(phases[j].imag)) if i == j else (0, 0)
            assert col[i] == want
    # exact back substitution in rationals
    Af = [[(Fraction(A[i, j].real), Fraction(A[i, j].imag)) for j in range(n)] for i in range(n)]
    bf = [(Fraction(v.real), Fraction(v.imag)) for v in b]

    def cmul(a, c):
        return (a[0] * c[0] - a[1] * c[1], a[0] * c[1] + a[1] * c[0])

    def cdiv(a, c):
        d = c[0] * c[0] + c[1] * c[1]
        return ((a[0] * c[0] + a[1] * c[1]) / d, (a[1] * c[0] - a[0] * c[1]) / d)

    x = [None] * n
    for k in range(n - 1, -1, -1):
        v = bf[k]
        for j in range(k + 1, n):
            p = cmul(Af[k][j], x[j])
            v = (v[0] - p[0], v[1] - p[1])
        x[k] = cdiv(v, Af[k][k])
    assert frac_vec(dx) == x
    assert rn == 0.0


def test_agrees_with_numpy_lstsq(orc):
    rng = np.random.default_rng(8)
    A = _rand_complex(rng, (10, 7))
    b = _rand_complex(rng, 10)
    st, dx, rn = orc.mgs_solve(_soa_mat(A, 2), soa_from_complex(b, 2))
    assert st == orc.OK
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    got = dx[0, 0] + 1j * dx[0, 1]
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref)) * np.linalg.cond(A)
    assert abs(rn - np.linalg.norm(A @ ref - b)) < 1e-12


def test_zero_column_is_nonfinite(orc):
    A = np.eye(4, dtype=complex)
    A[:, 2] = 0
    st, dx, rn = orc.mgs_solve(_soa_mat(A, 2), soa_from_complex(np.ones(4), 2))
    assert st == orc.NONFINITE
