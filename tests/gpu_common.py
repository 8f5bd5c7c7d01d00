"""Shared helpers of the GPU parity tests (numpy only: they must run where
mpmath is not installed).  Tolerances are relative to the sum of the
magnitudes of the terms of each output, the measure the accuracy targets are
stated in."""
from __future__ import annotations

import numpy as np

TOL_EVAL = {1: 1e-12, 2: 1e-28, 4: 1e-58}   # values and Jacobian, relative to sum |terms|
TOL_END = {1: 1e-10, 2: 1e-24, 4: 1e-52}    # path end points under the same schedule
U = {1: 2.0 ** -53, 2: 2.0 ** -104, 4: 2.0 ** -208}


def limb_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a - b for multi-limb arrays [L][...]: limb-wise differences summed
    from the leading limb (exact enough when a and b agree closely)."""
    d = np.zeros(a.shape[1:])
    for l in range(a.shape[0]):
        d = d + (a[l] - b[l])
    return d


def cabs_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """|a - b| for complex multi-limb arrays [L][2][...]."""
    d = limb_diff(a, b)
    return np.hypot(d[0], d[1])


def lead_complex(a: np.ndarray) -> np.ndarray:
    return a[0, 0] + 1j * a[0, 1]


def term_scale(spec, x: np.ndarray, t=None, gamma=None, k=1, g=None):
    """Sum of the magnitudes of the terms behind every output: (hs [N], Js [N, n])."""
    xa = np.abs(lead_complex(x))
    N, n = spec.N, spec.n

    def one(s):
        hs = np.zeros(N)
        Js = np.zeros((N, n))
        for i in range(N):
            for kk in range(s.term_ptr[i], s.term_ptr[i + 1]):
                vs = s.var_idx[s.var_ptr[kk]:s.var_ptr[kk + 1]]
                es = s.var_exp[s.var_ptr[kk]:s.var_ptr[kk + 1]]
                c = abs(s.coeff[kk])
                pw = xa[vs] ** es
                hs[i] += c * np.prod(pw)
                for q, (v, e) in enumerate(zip(vs, es)):
                    others = np.prod(pw[:q]) * np.prod(pw[q + 1:])
                    Js[i, v] += c * e * xa[v] ** (e - 1) * others
        return hs, Js

    hs, Js = one(spec)
    if gamma is None:
        return hs, Js
    sf = t ** k
    sg = (1 - t) ** k
    hs = sf * hs
    Js = sf * Js
    if g is not None:
        gh, gJ = one(g)
        return hs + sg * gh, Js + sg * gJ
    d = spec.degrees()
    for i in range(N):
        hs[i] += sg * (xa[i] ** d[i] + 1)
        Js[i, i] += sg * d[i] * xa[i] ** (d[i] - 1)
    return hs, Js


def assert_eval_close(L, spec, x, h_gpu, J_gpu, h_orc, J_orc, **hom):
    hs, Js = term_scale(spec, x, **hom)
    eh = cabs_diff(h_gpu, h_orc)
    eJ = cabs_diff(J_gpu, J_orc).T                # -> [N, n]
    tol = TOL_EVAL[L]
    rh = eh / np.maximum(hs, 1e-300)
    rJ = np.where(Js > 0, eJ / np.maximum(Js, 1e-300), eJ)
    assert rh.max() <= tol, f"value error {rh.max():.2e} > {tol:.0e}"
    assert rJ.max() <= tol, f"Jacobian error {rJ.max():.2e} > {tol:.0e}"
    return max(rh.max(), rJ.max())


def soa_from_complex(z, L: int) -> np.ndarray:
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    out = np.zeros((L, 2, len(z)))
    out[0, 0], out[0, 1] = z.real, z.imag
    return out


def soa_matrix(A, L: int) -> np.ndarray:
    """complex N x n (double) -> [L][2][n][N] column-major, zero-extended."""
    N, n = A.shape
    out = np.zeros((L, 2, n, N))
    out[0, 0] = A.T.real
    out[0, 1] = A.T.imag
    return out


def mgs_tol(A: np.ndarray, b: np.ndarray, L: int, c: float = 2.0) -> float:
    """Normwise bound on the difference of two backward-stable least-squares
    solutions of A x = b (A complex N x n, leading limbs) in L limbs:
    c n u (kappa + kappa^2 rho), rho = ||b - A x|| / (||A|| ||x||), the
    first-order forward error of least squares (the kappa^2 term vanishes
    for consistent systems), relative to ||x||_inf."""
    n = A.shape[1]
    s = np.linalg.svd(A, compute_uv=False)
    kappa = s[0] / s[-1]
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    rho = np.linalg.norm(b - A @ x) / (s[0] * np.linalg.norm(x))
    return c * n * U[L] * (kappa + kappa * kappa * rho)


def complex_matrix(J: np.ndarray) -> np.ndarray:
    """[L][2][n][N] -> complex N x n of the leading limbs."""
    return (J[0, 0] + 1j * J[0, 1]).T
