"""Pins of the oracle's evaluation of h(x,t) = gamma (1-t)^k g(x) + t^k f(x)
and its Jacobian (Section 2, Eq. (1)).

* Exact regime: small dyadic inputs make every product and sum exact in DD and
  QD, so the oracle must reproduce a brute-force evaluation in exact rationals
  bit for bit.  This catches any dropped term, wrong index, sign, exponent,
  transposed Jacobian or wrong homotopy factor.
* Accuracy: on random inputs the oracle agrees with a 300-bit mpmath
  evaluation to far below the DD/QD tolerances (relative to sum |terms|).
* Central differences in QD on DD points pin the Jacobian against the values
  (both real and imaginary directions, which catches a conjugation).
* Closed forms: cyclic n-roots (Section 4.2, Eq. (10)) at the all-ones point
  and at its root (1, w, w^2, ...), and the start system x_i^{d_i} - 1 at
  roots of unity.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1501_06625_gb300 import synth
from refmath import frac_vec, mp_vec, soa_from_complex, soa_from_mp

mpmath = pytest.importorskip("mpmath")


def _exact_eval(spec, x, t, gamma, k):
    """Brute force in exact complex rationals: x, gamma as (re, im) Fractions."""
    def cmul(a, b):
        return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])

    def cadd(a, b):
        return (a[0] + b[0], a[1] + b[1])

    def cpow(a, e):
        r = (Fraction(1), Fraction(0))
        for _ in range(e):
            r = cmul(r, a)
        return r

    N, n = spec.N, spec.n
    f = [(Fraction(0), Fraction(0))] * N
    Jf = [[(Fraction(0), Fraction(0))] * n for _ in range(N)]
    for i in range(N):
        for kk in range(spec.term_ptr[i], spec.term_ptr[i + 1]):
            c = (Fraction(spec.coeff[kk].real), Fraction(spec.coeff[kk].imag))
            vs = list(range(spec.var_ptr[kk], spec.var_ptr[kk + 1]))
            val = c
            for p in vs:
                val = cmul(val, cpow(x[spec.var_idx[p]], int(spec.var_exp[p])))
            f[i] = cadd(f[i], val)
            for q in vs:
                d = (c[0] * int(spec.var_exp[q]), c[1] * int(spec.var_exp[q]))
                for p in vs:
                    e = int(spec.var_exp[p]) - (1 if p == q else 0)
                    d = cmul(d, cpow(x[spec.var_idx[p]], e))
                j = spec.var_idx[q]
                Jf[i][j] = cadd(Jf[i][j], d)
    if gamma is None:
        return f, Jf
    deg = spec.degrees()
    tk = Fraction(t) ** k
    omtk = (1 - Fraction(t)) ** k
    sg = (gamma[0] * omtk, gamma[1] * omtk)
    h, J = [], [[None] * n for _ in range(N)]
    for i in range(N):
        gi = cadd(cpow(x[i], int(deg[i])), (Fraction(-1), Fraction(0)))
        h.append(cadd(cmul(sg, gi), (f[i][0] * tk, f[i][1] * tk)))
        for j in range(n):
            dg = (Fraction(0), Fraction(0))
            if i == j:
                dg = cmul((Fraction(int(deg[i])), Fraction(0)), cpow(x[i], int(deg[i]) - 1))
            J[i][j] = cadd(cmul(sg, dg), (Jf[i][j][0] * tk, Jf[i][j][1] * tk))
    return h, J


def _dyadic_system(seed, n, terms, nv, exps):
    rng = synth.Rng(seed)
    polys = []
    for _ in range(n):
        tl = []
        for _ in range(terms):
            vs = rng.sample(n, nv)
            c = [1, -1, 1j, -1j, 0.5 + 0.25j][rng.below(5)]
            tl.append((c, [(v, exps[rng.below(len(exps))]) for v in vs]))
        polys.append(tl)
    return synth.build_system(n, n, polys)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("seed,n,terms,nv,k", [(1, 3, 3, 2, 1), (2, 4, 4, 3, 2), (3, 5, 5, 2, 1)])
def test_exact_regime_bitwise(orc, L, seed, n, terms, nv, k):
    spec = _dyadic_system(seed, n, terms, nv, (1, 2))
    rng = np.random.default_rng(seed)
    xs = (rng.integers(-15, 16, n) + 1j * rng.integers(-15, 16, n)) / 16.0
    x = soa_from_complex(xs, L)
    t = 0.375
    gam = np.zeros((L, 2)); gam[0] = [0.375, 0.5]
    f = orc.System(spec, L)
    for gamma in (None, gam):
        h, J = orc.eval_h(f, x, t=t, gamma=gamma, k=k)
        xe = frac_vec(x)
        ge = None if gamma is None else (Fraction(gam[0, 0]), Fraction(gam[0, 1]))
        he, Je = _exact_eval(spec, xe, t, ge, k)
        got_h = frac_vec(h)
        assert got_h == he
        for j in range(n):
            col = frac_vec(J[:, :, j, :])
            assert col == [Je[i][j] for i in range(spec.N)]


def _mp_eval(spec, x, mp):
    f = [mp.mpc(0)] * spec.N
    scale = [mp.mpf(0)] * spec.N
    J = [[mp.mpc(0)] * spec.n for _ in range(spec.N)]
    Jscale = [[mp.mpf(0)] * spec.n for _ in range(spec.N)]
    for i in range(spec.N):
        for kk in range(spec.term_ptr[i], spec.term_ptr[i + 1]):
            c = mp.mpc(spec.coeff[kk].real, spec.coeff[kk].imag)
            vs = range(spec.var_ptr[kk], spec.var_ptr[kk + 1])
            val = c
            for p in vs:
                val *= x[spec.var_idx[p]] ** int(spec.var_exp[p])
            f[i] += val
            scale[i] += abs(val)
            for q in vs:
                d = c * int(spec.var_exp[q])
                for p in vs:
                    d *= x[spec.var_idx[p]] ** (int(spec.var_exp[p]) - (1 if p == q else 0))
                J[i][spec.var_idx[q]] += d
                Jscale[i][spec.var_idx[q]] += abs(d)
    return f, scale, J, Jscale


@pytest.mark.parametrize("L,tol", [(2, 1e-30), (4, 1e-61)])
def test_accuracy_vs_mpmath(orc, L, tol):
    mp = mpmath.mp
    mp.prec = 320
    rng = synth.Rng(7)
    spec = synth.dense_system(rng, 6, 6, 4, (1, 2, 3))
    xs = synth.random_x(rng, 6)
    x = soa_from_complex(xs, L)
    x[1] = x[0] * 2.0 ** -60            # a non-trivial second limb
    f = orc.System(spec, L)
    h, J = orc.eval_h(f, x)
    xm = mp_vec(x, mp)
    fe, sc, Je, Jsc = _mp_eval(spec, xm, mp)
    hm = mp_vec(h, mp)
    for i in range(spec.N):
        assert abs(hm[i] - fe[i]) / sc[i] < tol
        col = mp_vec(J[:, :, :, i], mp)
        for j in range(spec.n):
            if Jsc[i][j] > 0:
                assert abs(col[j] - Je[i][j]) / Jsc[i][j] < tol
            else:
                assert col[j] == 0


def test_central_differences_qd(orc):
    """J[:, j] against (f(x + s e_j) - f(x - s e_j)) / (2 s), s = 1e-20 real and
    imaginary, in QD on DD points: error O(s^2) + O(u_QD / s) ~ 1e-40."""
    L = 4
    rng = synth.Rng(9)
    spec = synth.dense_system(rng, 5, 5, 3, (1, 2, 3))
    xs = synth.random_x(rng, 5)
    x = soa_from_complex(xs, L)
    x[1] = x[0] * 2.0 ** -57
    f = orc.System(spec, L)
    _, J = orc.eval_h(f, x)
    mp = mpmath.mp
    mp.prec = 300
    s = 1e-20
    for j in range(spec.n):
        for part, unit in ((0, 1), (1, 1j)):
            xp = x.copy(); xp[2, part, j] = s
            xm = x.copy(); xm[2, part, j] = -s
            hp, _ = orc.eval_h(f, xp)
            hm_, _ = orc.eval_h(f, xm)
            dp, dm = mp_vec(hp, mp), mp_vec(hm_, mp)
            jc = mp_vec(J[:, :, j, :], mp)
            for i in range(spec.N):
                fd = (dp[i] - dm[i]) / (2 * s * unit)
                assert abs(fd - jc[i]) <= 1e-33 * (1 + abs(jc[i]))


@pytest.mark.parametrize("n", [5, 7])
def test_cyclic_closed_forms(orc, n):
    mp = mpmath.mp
    mp.prec = 300
    spec = synth.cyclic_system(n)
    for L in (2, 4):
        f = orc.System(spec, L)
        ones = soa_from_complex(np.ones(n), L)
        h, J = orc.eval_h(f, ones)
        hv = frac_vec(h)
        assert hv[:-1] == [(Fraction(n), Fraction(0))] * (n - 1)
        assert hv[-1] == (0, 0)
        for j in range(n):
            col = frac_vec(J[:, :, j, :])
            # variable j occurs in exactly i of the n products of i consecutive variables
            assert col == [(Fraction(i), Fraction(0)) for i in range(1, n)] + [(Fraction(1), Fraction(0))]
        # (1, w, w^2, ...) with w = exp(2 pi i / n) is a root for odd n
        w = [mp.expjpi(mp.mpf(2 * j) / n) for j in range(n)]
        xr = soa_from_mp(w, L, mp)
        h, _ = orc.eval_h(f, xr)
        u = 2.0 ** (-53 * L)
        assert max(abs(v) for v in mp_vec(h, mp)) < 50 * n * u


@pytest.mark.parametrize("L", [2, 4])
def test_start_system_roots_of_unity(orc, L):
    """h(x, 0) = gamma g(x) vanishes at x_i = exp(2 pi i m_i / d_i)."""
    mp = mpmath.mp
    mp.prec = 300
    rng = synth.Rng(5)
    spec = synth.dense_system(rng, 6, 4, 3, (1, 2, 3))
    deg = spec.degrees()
    f = orc.System(spec, L)
    for i in range(spec.n):
        assert f.degree(i) == deg[i]
    roots = [mp.expjpi(mp.mpf(2 * ((3 * i + 1) % int(deg[i]))) / int(deg[i])) for i in range(spec.n)]
    x = soa_from_mp(roots, L, mp)
    gam = np.zeros((L, 2)); gam[0] = [0.6, 0.8]
    h, J = orc.eval_h(f, x, t=0.0, gamma=gam)
    u = 2.0 ** (-53 * L)
    assert max(abs(v) for v in mp_vec(h, mp)) < 10 * max(deg) * u
    # at t = 0 the Jacobian is gamma * diag(d_i x_i^{d_i - 1})
    for j in range(spec.n):
        col = mp_vec(J[:, :, j, :], mp)
        expect = mp.mpc(0.6, 0.8) * int(deg[j]) * roots[j] ** (int(deg[j]) - 1)
        assert abs(col[j] - expect) < 10 * max(deg) * u * abs(expect)
        assert all(abs(col[i]) == 0 for i in range(spec.n) if i != j)


def test_homotopy_f_equals_g(orc):
    """When f is the start system itself, h = ((1-t) gamma + t) g vanishes on
    the start roots for every t."""
    L = 2
    n = 4
    polys = [[(1.0, [(i, 3)]), (-1.0, [])] for i in range(n)]
    spec = synth.build_system(n, n, polys)
    f = orc.System(spec, L)
    x = soa_from_complex(np.ones(n), L)
    gam = np.zeros((L, 2)); gam[0] = [0.75, -0.5]
    for t in (0.0, 0.25, 0.625, 1.0):
        h, J = orc.eval_h(f, x, t=t, gamma=gam)
        assert not np.any(h)
        d = frac_vec(J[:, :, 0, :])[0]
        # dh_0/dx_0 = 3 ((1-t) gamma + t) at x = 1
        tf = Fraction(t)
        assert d == ((1 - tf) * Fraction(0.75) * 3 + 3 * tf, (1 - tf) * Fraction(-0.5) * 3)


def test_rejects_bad_systems(orc):
    bad = synth.build_system(2, 2, [[(1.0, [(0, 1), (0, 2)])], [(1.0, [(1, 1)])]])
    with pytest.raises(ValueError):
        orc.System(bad, 2)
    bad = synth.build_system(2, 2, [[(1.0, [(2, 1)])], [(1.0, [(1, 1)])]])
    with pytest.raises(ValueError):
        orc.System(bad, 2)
