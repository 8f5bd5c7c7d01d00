"""The monodromy workload on cyclic n-roots (Section 4.2), n = m^2: its start
point must lie on the (m-1)-dimensional solution set that Backelin's lemma
gives, and the start slices must pass through it.

* the cyclic equations (Eq. (10)), evaluated in 60-digit arithmetic at the
  double start point, vanish to the rounding of that point;
* the Jacobian of the cyclic equations there has exactly m - 1 singular
  values at rounding level: the solution set has dimension m - 1 at x0, as
  many as there are slices;
* the oracle's evaluation of the start system [f; L] at x0 in double-double:
  the slice rows vanish to DD rounding (their constant terms are the exact
  sums stored as two limbs), the cyclic rows to the rounding of x0.
"""
import numpy as np
import pytest

import oracle
from paper_1501_06625_gb300 import synth

mpmath = pytest.importorskip("mpmath")


def _cyclic_mp(x):
    mp = mpmath.mp
    n = len(x)
    out = []
    for i in range(1, n):
        s = mp.mpc(0)
        for j in range(n):
            p = mp.mpc(1)
            for k in range(j, j + i):
                p *= x[k % n]
            s += p
        out.append(s)
    p = mp.mpc(1)
    for v in x:
        p *= v
    out.append(p - 1)
    return out


@pytest.mark.parametrize("n", [4, 9, 16])
def test_start_point_on_backelin_set(n):
    mpmath.mp.prec = 200
    F, G, gam, x0 = synth.cyclic_monodromy(3, n)
    xm = [mpmath.mpc(float(z.real), float(z.imag)) for z in x0]
    res = max(abs(v) for v in _cyclic_mp(xm))
    assert float(res) < 50 * n * 2.0 ** -53, float(res)


def _cyclic_jacobian(x):
    n = len(x)
    J = np.zeros((n, n), dtype=np.complex128)
    for i in range(1, n):                       # f_i: windows of length i
        for j in range(n):
            idx = [(j + k) % n for k in range(i)]
            for q in idx:
                J[i - 1, q] += np.prod([x[r] for r in idx if r != q])
    for q in range(n):
        J[n - 1, q] = np.prod([x[r] for r in range(n) if r != q])
    return J


@pytest.mark.parametrize("m", [2, 3, 4])
def test_solution_set_dimension(m):
    n = m * m
    _, _, _, x0 = synth.cyclic_monodromy(5, n)
    s = np.linalg.svd(_cyclic_jacobian(x0), compute_uv=False)
    assert np.all(s[-(m - 1):] < 1e-11 * s[0]), s
    assert s[-m] > 1e-4 * s[0], s


@pytest.mark.parametrize("L", [2, 4])
def test_start_slices_pass_through_x0(L):
    n, m = 16, 4
    F, G, gam, x0 = synth.cyclic_monodromy(1, n, fixed=False)      # G = [f; L]
    assert (F.N, F.n, G.N) == (n + m - 1, n, n + m - 1)
    xs = np.zeros((L, 2, n))
    xs[0, 0], xs[0, 1] = x0.real, x0.imag
    h, _ = oracle.eval_h(oracle.System(G, L), xs)
    hv = h[0, 0] + 1j * h[0, 1]
    assert np.abs(hv[:n]).max() < 50 * n * 2.0 ** -53
    # the slice rows: DD/QD evaluation of an exact sum: rounding of DD only
    assert np.abs(hv[n:]).max() < 1e-28
    h, _ = oracle.eval_h(oracle.System(F, L), xs)
    assert np.abs(h[0, 0, n:] + 1j * h[0, 1, n:]).min() > 1e-3     # K does not


@pytest.mark.parametrize("L", [2, 4])
def test_fixed_rows_homotopy(L):
    """With fixed rows the oracle evaluates the paper's monodromy homotopy
    [f; gamma (1-t) L + t K] for F = [f; K], G = [0; L]: the cyclic rows are
    f's own values and derivatives in every limb (not scaled by t), the slice
    rows the combination of the two slices; without fixed rows the cyclic rows
    are t f (G has no terms there)."""
    n = 16
    F, G, gam, _ = synth.cyclic_monodromy(2, n)
    x = np.zeros((L, 2, n))
    z = synth.random_x(synth.Rng(9), n)
    x[0, 0], x[0, 1] = z.real, z.imag
    gs = np.zeros((L, 2))
    gs[0] = [gam.real, gam.imag]
    t = 0.37
    oF, oG = oracle.System(F, L), oracle.System(G, L)
    h, J = oracle.eval_h(oF, x, t=t, gamma=gs, g=oG, fixed_rows=1)
    hF, JF = oracle.eval_h(oF, x)
    hG, _ = oracle.eval_h(oG, x)
    assert np.array_equal(h[:, :, :n], hF[:, :, :n])
    assert np.array_equal(J[:, :, :, :n], JF[:, :, :, :n])

    def lead(a):
        return a[0, 0] + 1j * a[0, 1]

    want = gam * (1 - t) * lead(hG)[n:] + t * lead(hF)[n:]
    assert np.abs(lead(h)[n:] - want).max() < 1e-14 * np.abs(want).max()
    h0, _ = oracle.eval_h(oF, x, t=t, gamma=gs, g=oG, fixed_rows=0)
    ref = np.abs(lead(hF)[:n]).max()
    assert np.abs(lead(h0)[:n] - t * lead(hF)[:n]).max() < 1e-14 * ref


def _slices(spec, n, m):
    """coefficients and constants of the slice rows of a start system [0; L]"""
    r = m - 1
    c = spec.coeff.reshape(r, n + 1)
    lo = spec.coeff_lo.reshape(r, n + 1)[:, n]
    return c[:, :n], c[:, n] + lo


def _cyclic_np(x):
    n = len(x)
    out = [sum(np.prod([x[(j + k) % n] for k in range(i)]) for j in range(n)) for i in range(1, n)]
    return np.array(out + [np.prod(x) - 1])


@pytest.mark.parametrize("m", [2, 3, 4])
def test_family_points_on_the_slices(m):
    """The m points of Backelin's family on the start slices, computed from the
    linear parametrization: they satisfy the cyclic equations and the slices,
    are distinct, and the start point is one of them."""
    from paper_1501_06625_gb300 import monodromy
    n = m * m
    loop = synth.cyclic_monodromy_loop(4, n)
    coef, const = _slices(loop["out"][1], n, m)
    pts = monodromy.family_points_on_slices(m, coef, const)
    assert pts.shape == (m, n)
    for x in pts:
        assert np.abs(_cyclic_np(x)).max() < 1e-10 * max(1.0, np.abs(x).max() ** n)
        assert np.abs(coef @ x + const).max() < 1e-12 * np.abs(coef).sum(axis=1).max() * np.abs(x).max()
    d = np.abs(pts[:, None, :] - pts[None, :, :]).max(axis=2) + np.eye(m)
    assert d.min() > 1e-6
    assert np.abs(pts - loop["x0"][None, :]).max(axis=1).min() < 1e-12


def test_loop_halves_swap_the_slices():
    """The way back moves K to L: its target carries the start system's slices
    L (with their two-limb constants) after the cyclic rows, its start system
    the target's slices K with empty cyclic rows; the way out is the fixed-row
    form of cyclic_monodromy."""
    n, m = 16, 4
    r = m - 1
    loop = synth.cyclic_monodromy_loop(6, n)
    F, G = loop["out"]
    Fb, Gb = loop["back"]
    F0, G0, _, x0 = synth.cyclic_monodromy(6, n)
    assert np.array_equal(F.coeff, F0.coeff) and np.array_equal(G.coeff, G0.coeff)
    assert np.array_equal(x0, loop["x0"])
    k = r * (n + 1)
    assert np.array_equal(Fb.coeff[-k:], G.coeff[-k:])
    assert np.array_equal(Fb.coeff_lo[-k:], G.coeff_lo[-k:])
    assert np.array_equal(Gb.coeff, F.coeff[-k:])
    assert np.array_equal(Fb.coeff[:-k], F.coeff[:-k])          # the cyclic rows
    assert (Gb.term_ptr[:n + 1] == 0).all() and (G.term_ptr[:n + 1] == 0).all()
    assert Fb.N == Gb.N == F.N == n + r


def test_oracle_monodromy_loops_find_the_degree():
    """The oracle alone, with the cyclic rows held fixed, runs monodromy loops
    on cyclic 4-roots (m = 2): out to the slices K and back to L with random
    alpha and beta, from the points found so far.  It finds the m = 2 points of
    the component on L, each equal to a point of the family's linear
    parametrization, and no other."""
    from paper_1501_06625_gb300 import monodromy
    n, m, L = 4, 2, 2
    loop = synth.cyclic_monodromy_loop(2, n)
    F, G = loop["out"]
    Fb, Gb = loop["back"]
    oF, oG, oFb, oGb = (oracle.System(s, L) for s in (F, G, Fb, Gb))
    rng = synth.Rng(11)
    p = synth.default_params(L, max_newton=5, max_steps=3000, fixed_rows=1)
    x0 = np.zeros((L, 2, n))
    x0[0, 0], x0[0, 1] = loop["x0"].real, loop["x0"].imag
    pts = [x0]
    for i in range(6):
        ga, gb = np.zeros((L, 2)), np.zeros((L, 2))
        a, b = rng.unit_complex(), rng.unit_complex()
        ga[0], gb[0] = [a.real, a.imag], [b.real, b.imag]
        st, y, _, _ = oracle.track(oF, pts[i % len(pts)], ga, p, g=oG)
        assert st == oracle.OK
        st, z, _, _ = oracle.track(oFb, y, gb, p, g=oGb)
        assert st == oracle.OK
        zl = z[0, 0] + 1j * z[0, 1]
        if all(np.abs(zl - (q[0, 0] + 1j * q[0, 1])).max() > 1e-8 for q in pts):
            pts.append(z)
    assert len(pts) == m
    c = G.coeff.reshape(m - 1, n + 1)
    ref = monodromy.family_points_on_slices(
        m, c[:, :n], c[:, n] + G.coeff_lo.reshape(m - 1, n + 1)[:, n])
    for q in pts:
        assert np.abs(ref - (q[0, 0] + 1j * q[0, 1])[None, :]).max(axis=1).min() < 1e-12
