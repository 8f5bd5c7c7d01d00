"""Pins of the oracle's mixed-precision corrector (oracle/mixed.c) against
references that do not use it:

* the low-precision MGS solve against LAPACK least squares (numpy.linalg.lstsq)
  within the backward-stable forward error bound of its precision, for square
  and overdetermined systems; its condition estimate against the singular
  values (it is a lower bound of the 2-norm condition number);
* the mixed corrector on a linear target, iterated, against the exact solution
  (400-bit mpmath LU): the error contracts by about kappa u_low per iteration
  and ends at working precision, which shows the update accumulates in DD/QD;
* the mixed corrector on x^3 = c against the closed-form cube root;
* a zero column is reported, not divided by.
"""
import numpy as np
import pytest

from paper_1501_06625_gb300 import synth
from refmath import mp_vec, soa_from_complex

mpmath = pytest.importorskip("mpmath")

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


def _random_system(rng, N, n, cond):
    """A complex N x n matrix with singular values log-spaced in [1/cond, 1]."""
    def unitary(m):
        q, r = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
        return q * (np.diag(r) / np.abs(np.diag(r)))
    s = np.logspace(0, -np.log10(cond), n)
    A = unitary(N)[:, :n] @ np.diag(s) @ unitary(n).conj().T
    return A, s


@pytest.mark.parametrize("lin", ["f64", "f32"])
@pytest.mark.parametrize("N,n", [(6, 6), (12, 12), (20, 13)])
def test_lowprec_solve_against_lstsq(orc, lin, N, n):
    rng = np.random.default_rng(N * 100 + n)
    cond = 1e3 if lin == "f32" else 1e8
    A, s = _random_system(rng, N, n, cond)
    xt = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b = A @ xt
    if N > n:                                   # a component outside the range
        b = b + 1e-3 * (np.eye(N) - A @ np.linalg.pinv(A)) @ (rng.standard_normal(N) + 0j)
    st, x, est = orc.lowprec_solve(A, b, lin)
    assert st == orc.OK
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    kappa = s[0] / s[-1]
    err = np.abs(x - ref).max() / np.abs(ref).max()
    # least-squares forward error: kappa u + kappa^2 u |r| / (|A| |x|)
    r = np.linalg.norm(b - A @ ref) / (s[0] * np.linalg.norm(ref))
    assert err <= 30 * n * U[lin] * (kappa + kappa ** 2 * r), (err, kappa)
    # a lower bound of the condition number, not below 1
    assert 1.0 <= est <= kappa * (1 + 1e-3)


@pytest.mark.parametrize("lin", ["f64", "f32"])
def test_lowprec_solve_zero_column(orc, lin):
    A = np.eye(4, dtype=complex)
    A[:, 2] = 0
    st, _, _ = orc.lowprec_solve(A, np.ones(4), lin)
    assert st == orc.NONFINITE


def _linear_target(rng, n):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 2 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    polys = [[(A[i, j], [(j, 1)]) for j in range(n)] + [(-b[i], [])] for i in range(n)]
    return A, b, synth.build_system(n, n, polys)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("lin", ["f64", "f32"])
def test_mixed_corrector_linear_target(orc, L, lin):
    """On f = Ax - b at t = 1 the mixed corrector is iterative refinement:
    each iteration multiplies the error by about kappa u_low, down to working
    precision (which a double-precision update could not reach)."""
    mp = mpmath.mp
    mp.prec = 400
    n = 5
    rng = np.random.default_rng(3)
    A, b, spec = _linear_target(rng, n)
    f = orc.System(spec, L)
    Am = mp.matrix([[mp.mpc(A[i, j].real, A[i, j].imag) for j in range(n)] for i in range(n)])
    bm = mp.matrix([mp.mpc(v.real, v.imag) for v in b])
    xs = mp.lu_solve(Am, bm)
    gam = np.zeros((L, 2)); gam[0] = [0.6, 0.8]
    x = soa_from_complex(np.zeros(n), L)
    kappa = np.linalg.cond(A)
    rate = 30 * n * kappa * U[lin]
    uL = 2.0 ** (-53 * L)
    errs = []
    for _ in range(40):
        _, x, it, upd, res, dxn, est = orc.newton_mixed(
            f, x, 1.0, gam, synth.default_params(L, max_newton=1), lin, fixed=True)
        assert it == 1 and upd == 1
        got = mp_vec(x, mp)
        errs.append(float(max(abs(got[i] - xs[i]) for i in range(n)) / max(abs(v) for v in xs)))
        if errs[-1] < 10 * uL:
            break
    assert errs[-1] < 100 * kappa * uL, errs
    for a, c in zip(errs, errs[1:]):            # contraction until the floor
        assert c <= max(rate * a, 100 * kappa * uL), errs
    assert 1.0 <= est <= kappa * (1 + 1e-6)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("lin", ["f64", "f32"])
def test_mixed_corrector_cube_root(orc, L, lin):
    mp = mpmath.mp
    mp.prec = 400
    c = 0.3 + 0.4j
    spec = synth.build_system(1, 1, [[(1.0, [(0, 3)]), (-c, [])]])
    f = orc.System(spec, L)
    gam = np.zeros((L, 2)); gam[0] = [0.6, 0.8]
    w = mp.mpc(c.real, c.imag) ** (mp.mpf(1) / 3)
    start = soa_from_complex([complex(w) * (1 + 1e-4)], L)
    uL = 2.0 ** (-53 * L)
    params = synth.default_params(L, max_newton=40)
    ok, x, it, upd, res, dxn, est = orc.newton_mixed(f, start, 1.0, gam, params, lin)
    assert ok
    # the corrector stops once the residual or the update is below tolerance ...
    assert abs(mp_vec(x, mp)[0] - w) < 10 * max(params["tol_res"], params["tol_dx"])
    # ... and a few more iterations reach working precision
    _, xr, *_ = orc.newton_mixed(f, x, 1.0, gam, dict(params, max_newton=3), lin, fixed=True)
    assert abs(mp_vec(xr, mp)[0] - w) < 100 * uL
    # at most a few more iterations than the all-working-precision corrector
    ok2, x2, it2, *_ = orc.newton(f, start, 1.0, gam, params)
    assert ok2 and it <= it2 + (4 if lin == "f64" else 12)
    assert abs(est - 1.0) < 1e-6                 # a 1 x 1 system: r_00 / r_00


def test_planted_root_is_exact(orc):
    """The planted generator's constant terms make f(x*) = 0 exactly: checked
    by evaluating every polynomial at x* in rationals, and by the oracle."""
    from fractions import Fraction
    rng = synth.Rng(9)
    spec, xs = synth.planted_system(rng, 6, 7, 3, (1, 2, 3), 12.0)
    for i in range(spec.N):
        sre, sim = Fraction(0), Fraction(0)
        for k in range(spec.term_ptr[i], spec.term_ptr[i + 1]):
            cre = Fraction(spec.coeff[k].real) + Fraction(spec.coeff_lo[k].real)
            cim = Fraction(spec.coeff[k].imag) + Fraction(spec.coeff_lo[k].imag)
            ure, uim = Fraction(1), Fraction(0)
            for q in range(spec.var_ptr[k], spec.var_ptr[k + 1]):
                z = xs[spec.var_idx[q]]
                for _ in range(int(spec.var_exp[q])):
                    ure, uim = ure * Fraction(z.real) - uim * Fraction(z.imag), \
                        ure * Fraction(z.imag) + uim * Fraction(z.real)
            sre += cre * ure - cim * uim
            sim += cre * uim + cim * ure
        assert sre == 0 and sim == 0
    for i in range(spec.N):                     # moduli in [1e-12, 1], the largest 1
        ks = [k for k in range(spec.term_ptr[i], spec.term_ptr[i + 1])
              if spec.var_ptr[k + 1] > spec.var_ptr[k]]
        m = np.abs(spec.coeff[ks])
        assert abs(m.max() - 1.0) < 1e-15 and m.min() >= 1e-12 * (1 - 1e-15)
    for L in (2, 4):
        h, _ = orc.eval_h(orc.System(spec, L), soa_from_complex(xs, L), t=1.0)
        assert not np.any(h)


def test_sparse_planted_root_is_exact(orc):
    """The sparse planted generator (the sparse n = 512 recipe with a planted
    root, here at n = 40): f(x*) = 0 exactly in rationals and by the oracle,
    and every polynomial keeps the recipe's linear term in its own variable."""
    from fractions import Fraction
    rng = synth.Rng(11)
    spec, xs = synth.sparse_planted(rng, 40)
    for i in range(spec.N):
        sre, sim = Fraction(0), Fraction(0)
        for k in range(spec.term_ptr[i], spec.term_ptr[i + 1]):
            cre = Fraction(spec.coeff[k].real) + Fraction(spec.coeff_lo[k].real)
            cim = Fraction(spec.coeff[k].imag) + Fraction(spec.coeff_lo[k].imag)
            ure, uim = Fraction(1), Fraction(0)
            for q in range(spec.var_ptr[k], spec.var_ptr[k + 1]):
                z = xs[spec.var_idx[q]]
                for _ in range(int(spec.var_exp[q])):
                    ure, uim = ure * Fraction(z.real) - uim * Fraction(z.imag), \
                        ure * Fraction(z.imag) + uim * Fraction(z.real)
            sre += cre * ure - cim * uim
            sim += cre * uim + cim * ure
        assert sre == 0 and sim == 0
        k0 = spec.term_ptr[i]                       # the linear term c x_i comes first
        assert list(spec.var_idx[spec.var_ptr[k0]:spec.var_ptr[k0 + 1]]) == [i]
        assert list(spec.var_exp[spec.var_ptr[k0]:spec.var_ptr[k0 + 1]]) == [1]
    for L in (2, 4):
        h, _ = orc.eval_h(orc.System(spec, L), soa_from_complex(xs, L), t=1.0)
        assert not np.any(h)
