"""Seeded synthetic workloads for the path tracker.

This module holds the input generators that both the CUDA library's tests and
benchmarks and the CPU oracle consume.  It contains no arithmetic of the method
itself: only pseudo-random draws, the combinatorial structure of the systems
(supports and exponents) and unit-modulus coefficients rounded to double.

Random numbers come from xoshiro256** seeded through splitmix64, both written
here from their published definitions (Blackman & Vigna, "Scrambled linear
pseudorandom number generators", 2018), so every run on every machine draws the
same systems from the same seed.

The paper's benchmark inputs (Pieri systems, cyclic n-roots start points,
Section 4) came from scripts that are not available; the workloads below stand
in for them by shape: dense general polynomials below dimension 100 (where
evaluation and differentiation dominate, Introduction) and very sparse
low-degree systems of several hundred equations (where the linear algebra
dominates, Introduction).  The cyclic n-roots system (Section 4.2) has a closed
form and is generated exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & _MASK


class Rng:
    """xoshiro256** with splitmix64 seeding."""

    def __init__(self, seed: int):
        z = seed & _MASK
        self.s = []
        for _ in range(4):
            z = (z + 0x9E3779B97F4A7C15) & _MASK
            w = z
            w = ((w ^ (w >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
            w = ((w ^ (w >> 27)) * 0x94D049BB133111EB) & _MASK
            self.s.append(w ^ (w >> 31))

    def next_u64(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & _MASK, 7) * 9) & _MASK
        t = (s[1] << 17) & _MASK
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self) -> float:
        """53-bit uniform in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, m: int) -> int:
        """Integer in [0, m) by multiply-shift of a 64-bit draw."""
        return (self.next_u64() * m) >> 64

    def choice(self, seq):
        return seq[self.below(len(seq))]

    def sample(self, n: int, k: int) -> list[int]:
        """k distinct integers of range(n), partial Fisher-Yates, sorted."""
        if k > n:
            raise ValueError("sample larger than population")
        pool = list(range(n))
        for i in range(k):
            j = i + self.below(n - i)
            pool[i], pool[j] = pool[j], pool[i]
        return sorted(pool[:k])

    def unit_complex(self) -> complex:
        """e^{i theta}, theta = 2 pi u, rounded to double."""
        th = 2.0 * math.pi * self.uniform()
        return complex(math.cos(th), math.sin(th))


@dataclass
class SystemSpec:
    """A fully expanded polynomial system: N polynomials in n variables.

    Polynomial i owns terms term_ptr[i]..term_ptr[i+1]-1; term k owns the
    (variable, exponent) pairs var_ptr[k]..var_ptr[k+1]-1 (exponent >= 1, the
    variables of a term distinct); a term with no pair is a constant.
    coeff[k] is the complex coefficient of term k, a double; coeff_lo, when
    given, holds a second limb (a coefficient is then coeff + coeff_lo
    exactly, which a planted constant term needs).
    """

    N: int
    n: int
    term_ptr: np.ndarray
    var_ptr: np.ndarray
    var_idx: np.ndarray
    var_exp: np.ndarray
    coeff: np.ndarray
    coeff_lo: np.ndarray | None = None

    @property
    def M(self) -> int:
        return int(self.term_ptr[-1])

    def coeff_soa(self, L: int) -> np.ndarray:
        """Coefficients as [L][2][M] doubles, zero-extended to L limbs."""
        out = np.zeros((L, 2, self.M))
        out[0, 0] = self.coeff.real
        out[0, 1] = self.coeff.imag
        # in one limb a two-limb coefficient is its leading limb, which is its
        # correctly rounded double
        if self.coeff_lo is not None and L >= 2:
            out[1, 0] = self.coeff_lo.real
            out[1, 1] = self.coeff_lo.imag
        return out

    def degrees(self) -> np.ndarray:
        d = np.zeros(self.N, dtype=np.int64)
        for i in range(self.N):
            for k in range(self.term_ptr[i], self.term_ptr[i + 1]):
                d[i] = max(d[i], int(self.var_exp[self.var_ptr[k]:self.var_ptr[k + 1]].sum()))
        return d

    def max_vars(self) -> int:
        return int(np.diff(self.var_ptr).max()) if self.M else 0


def build_system(N: int, n: int, polys: list[list[tuple[complex, list[tuple[int, int]]]]]) -> SystemSpec:
    """polys[i] = list of (coefficient, [(var, exp), ...]) terms."""
    term_ptr, var_ptr, var_idx, var_exp, coeff = [0], [0], [], [], []
    for terms in polys:
        for c, mono in terms:
            coeff.append(complex(c))
            for v, e in mono:
                var_idx.append(v)
                var_exp.append(e)
            var_ptr.append(len(var_idx))
        term_ptr.append(len(coeff))
    return SystemSpec(N, n,
                      np.asarray(term_ptr, dtype=np.int32), np.asarray(var_ptr, dtype=np.int32),
                      np.asarray(var_idx, dtype=np.int32), np.asarray(var_exp, dtype=np.int32),
                      np.asarray(coeff, dtype=np.complex128))


def dense_system(rng: Rng, n: int, terms_per_poly: int, vars_per_term: int,
                 exps: tuple[int, ...], log10_mag: float = 0.0) -> SystemSpec:
    """Each polynomial: terms over `vars_per_term` distinct variables drawn
    uniformly without replacement, exponents uniform in `exps`, coefficients of
    unit modulus (or modulus 10^{U[0, log10_mag]}) and uniform angle."""
    polys = []
    for _ in range(n):
        terms = []
        for _ in range(terms_per_poly):
            vs = rng.sample(n, vars_per_term)
            mono = [(v, rng.choice(exps)) for v in vs]
            c = rng.unit_complex()
            if log10_mag > 0.0:
                c = c * 10.0 ** (log10_mag * rng.uniform())
            terms.append((c, mono))
        polys.append(terms)
    return build_system(n, n, polys)


def sparse_system(rng: Rng, n: int, extra_terms: int = 3, vars_per_term: int = 2,
                  exps: tuple[int, ...] = (1, 2)) -> SystemSpec:
    """Polynomial i: a linear term c x_i plus `extra_terms` monomials over
    `vars_per_term` distinct variables other than x_i, exponents in `exps`."""
    polys = []
    for i in range(n):
        terms = [(rng.unit_complex(), [(i, 1)])]
        for _ in range(extra_terms):
            vs = rng.sample(n - 1, vars_per_term)
            vs = [v if v < i else v + 1 for v in vs]
            terms.append((rng.unit_complex(), [(v, rng.choice(exps)) for v in vs]))
        polys.append(terms)
    return build_system(n, n, polys)


def planted_system(rng: Rng, n: int, terms_per_poly: int, vars_per_term: int,
                   exps: tuple[int, ...], log10_mag: float,
                   per_equation: bool = False) -> tuple[SystemSpec, np.ndarray]:
    """A dense system (the recipe of dense_system) whose coefficient moduli
    spread log-uniformly over log10_mag decades within each polynomial, with a
    planted root x*.  Each polynomial is scaled so that its largest modulus is
    1: the moduli are 10^{log10_mag (u - u_max)}, u uniform.  (Unscaled moduli up
    to 10^log10_mag against the unit-size start system would put a boundary
    layer of width ~10^-log10_mag at t = 0 that no step size crosses; scaling
    an equation changes neither its roots nor the spread within it.)  Each
    coordinate of x* is drawn from {1, i, -1, -i}, so every term's value
    c (x*)^a is c with its parts swapped or negated, exactly; each polynomial
    gets the constant term b_i = -sum_k c_ik (x*)^{a_ik}, summed exactly in
    rationals and stored as two limbs, so f(x*) = 0 holds exactly.
    With per_equation, the spread is between the equations instead: every
    term of polynomial i has modulus 10^{log10_mag u_i} (one draw u_i per
    polynomial, no rescaling), so the rows of the Jacobian differ in scale by
    up to 10^log10_mag and its condition number grows with them.
    Returns (system, x*)."""
    from fractions import Fraction
    units = (1 + 0j, 1j, -1 + 0j, -1j)
    xs = np.array([rng.choice(units) for _ in range(n)])
    polys, lo = [], []
    for _ in range(n):
        drawn = []
        for _ in range(terms_per_poly):
            vs = rng.sample(n, vars_per_term)
            mono = [(v, rng.choice(exps)) for v in vs]
            drawn.append((mono, rng.unit_complex(), rng.uniform()))
        umax = max(u for _, _, u in drawn)
        if per_equation:
            ue = rng.uniform()
            drawn = [(mono, e, ue) for mono, e, _ in drawn]
            umax = 0.0
        terms = []
        bre, bim = Fraction(0), Fraction(0)
        for mono, e, u in drawn:
            c = e * 10.0 ** (log10_mag * (u - umax))
            w = c
            for v, k in mono:
                w = w * xs[v] ** k                 # exact: a swap or negation of parts
            bre -= Fraction(w.real)
            bim -= Fraction(w.imag)
            terms.append((c, mono))
            lo.append(0j)
        hre, him = float(bre), float(bim)
        lre, lim = float(bre - Fraction(hre)), float(bim - Fraction(him))
        if Fraction(hre) + Fraction(lre) != bre or Fraction(him) + Fraction(lim) != bim:
            raise ValueError("the constant term does not fit in two limbs")
        terms.append((complex(hre, him), []))
        lo.append(complex(lre, lim))
        polys.append(terms)
    spec = build_system(n, n, polys)
    spec.coeff_lo = np.asarray(lo, dtype=np.complex128)
    return spec, xs


def sparse_planted(rng: Rng, n: int, extra_terms: int = 3, vars_per_term: int = 2,
                   exps: tuple[int, ...] = (1, 2)) -> tuple[SystemSpec, np.ndarray]:
    """The sparse recipe of sparse_system (a linear term c x_i plus
    `extra_terms` monomials over `vars_per_term` other variables) with a
    planted root x*: coordinates drawn from {1, i, -1, -i}, and polynomial i
    gets the constant term b_i = -sum_k c_ik (x*)^{a_ik}, summed exactly in
    rationals and stored as two limbs, so that f(x*) = 0 exactly.  Returns
    (system, x*)."""
    from fractions import Fraction
    units = (1 + 0j, 1j, -1 + 0j, -1j)
    xs = np.array([rng.choice(units) for _ in range(n)])
    polys, lo = [], []
    for i in range(n):
        drawn = [(rng.unit_complex(), [(i, 1)])]
        for _ in range(extra_terms):
            vs = rng.sample(n - 1, vars_per_term)
            vs = [v if v < i else v + 1 for v in vs]
            drawn.append((rng.unit_complex(), [(v, rng.choice(exps)) for v in vs]))
        terms = []
        bre, bim = Fraction(0), Fraction(0)
        for c, mono in drawn:
            w = c
            for v, k in mono:
                w = w * xs[v] ** k                 # exact: a swap or negation of parts
            bre -= Fraction(w.real)
            bim -= Fraction(w.imag)
            terms.append((c, mono))
            lo.append(0j)
        hre, him = float(bre), float(bim)
        lre, lim = float(bre - Fraction(hre)), float(bim - Fraction(him))
        if Fraction(hre) + Fraction(lre) != bre or Fraction(him) + Fraction(lim) != bim:
            raise ValueError("the constant term does not fit in two limbs")
        terms.append((complex(hre, him), []))
        lo.append(complex(lre, lim))
        polys.append(terms)
    spec = build_system(n, n, polys)
    spec.coeff_lo = np.asarray(lo, dtype=np.complex128)
    return spec, xs


def cyclic_system(n: int) -> SystemSpec:
    """Cyclic n-roots (Section 4.2, Eq. (10)): f_i = sum_j prod_{k=j}^{j+i-1}
    x_{k mod n} for i = 1..n-1, and f_n = x_0 x_1 ... x_{n-1} - 1.  Built with
    array operations: n = 352 has about 21.7 million (variable, exponent)
    pairs.  The variables of each term are listed in increasing order."""
    if n < 2:
        raise ValueError("cyclic n-roots needs n >= 2")
    lengths = [np.full(n, i, dtype=np.int64) for i in range(1, n)]
    lengths.append(np.array([n, 0], dtype=np.int64))          # x_0..x_{n-1}, then -1
    tl = np.concatenate(lengths)                               # variables per term
    M = tl.size
    var_ptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(tl, out=var_ptr[1:])
    var_idx = np.empty(int(var_ptr[-1]), dtype=np.int32)
    pos = 0
    for i in range(1, n):                                      # terms of f_i: windows of i
        j = np.arange(n)[:, None]
        win = (j + np.arange(i)[None, :]) % n
        win.sort(axis=1)
        var_idx[pos:pos + n * i] = win.ravel()
        pos += n * i
    var_idx[pos:pos + n] = np.arange(n)
    term_ptr = np.zeros(n + 1, dtype=np.int64)
    term_ptr[1:n] = n * np.arange(1, n)
    term_ptr[n] = M
    coeff = np.ones(M, dtype=np.complex128)
    coeff[-1] = -1.0
    return SystemSpec(n, n, term_ptr.astype(np.int32), var_ptr.astype(np.int32), var_idx,
                      np.ones(var_idx.size, dtype=np.int32), coeff)


def backelin_point(m: int, v: np.ndarray) -> np.ndarray:
    """A point of the (m-1)-dimensional solution set of cyclic n-roots,
    n = m^2, that Backelin's lemma asserts (Section 4.2).  Writing
    x_k = z_{k+1} / z_k (indices mod n) turns f_i = 0 (i < n) into the vanishing
    of the periodic correlations sum_j z_{j+i} / z_j, and makes f_n = 0 read
    prod x_k = 1, which then holds.  The sequence z_{am+b} = w^{ab} u_b
    (0 <= a, b < m, w = e^{2 pi i/m}, u_b free) has every correlation zero: the
    sum over a kills each shift that is not a multiple of m, the sum over b
    each that is.  In x this is x_{am+b} = w^a v_b with v_b = u_{b+1} / u_b, that
    is, any v with prod_b v_b = 1: v gives the m - 1 free parameters.
    v: m complex numbers; v[m-1] is replaced by 1 / prod(v[:m-1])."""
    v = np.asarray(v, dtype=np.complex128).copy()
    v[m - 1] = 1.0 / np.prod(v[:m - 1])
    a = np.arange(m)
    w = np.exp(2j * np.pi * a / m)
    return (w[:, None] * v[None, :]).ravel()              # index a m + b


def _with_linear_rows(spec: SystemSpec, coef: np.ndarray, const: np.ndarray,
                      const_lo: np.ndarray) -> SystemSpec:
    """spec followed by the rows sum_k coef[r, k] x_k + const[r] (+ const_lo[r],
    a second limb)."""
    r, n = coef.shape
    M0 = spec.M
    term_ptr = np.concatenate([spec.term_ptr.astype(np.int64),
                               M0 + (n + 1) * np.arange(1, r + 1)])
    lens = np.tile(np.append(np.ones(n, dtype=np.int64), 0), r)
    var_ptr = np.concatenate([spec.var_ptr.astype(np.int64),
                              spec.var_ptr[-1] + np.cumsum(lens)])
    var_idx = np.concatenate([spec.var_idx, np.tile(np.arange(n, dtype=np.int32), r)])
    var_exp = np.concatenate([spec.var_exp, np.ones(n * r, dtype=np.int32)])
    coeff = np.concatenate([spec.coeff, np.hstack([coef, const[:, None]]).ravel()])
    lo0 = spec.coeff_lo if spec.coeff_lo is not None else np.zeros(M0, dtype=np.complex128)
    lo = np.concatenate([lo0, np.hstack([np.zeros((r, n)), const_lo[:, None]]).ravel()])
    return SystemSpec(spec.N + r, spec.n, term_ptr.astype(np.int32), var_ptr.astype(np.int32),
                      var_idx.astype(np.int32), var_exp.astype(np.int32), coeff,
                      lo.astype(np.complex128))


def cyclic_monodromy(seed: int, n: int, fixed: bool = True):
    """One monodromy path on cyclic n-roots, n = m^2 (Section 4.2): the
    solution set of dimension m - 1 cut by m - 1 random hyperplanes L, moved to
    m - 1 other random hyperplanes K: N = n + m - 1 equations in n unknowns,
    corrected by least squares.  fixed: F = [f; K] and G = [0; L], the paper's
    homotopy {f = 0, alpha (1-t) L + t K = 0} when the tracker holds the rows
    without a start term fixed (ph_track_params.fixed_rows = 1, gamma =
    alpha).  Otherwise G = [f; L]: gamma (1-t) G + t F has the same zero set
    (its first block is f times gamma (1-t) + t, which does not vanish for t in
    [0, 1]) and evaluates f twice.  The start point is backelin_point with v of
    unit modulus (random angles); L's constant terms are -sum_k c_k x0_k,
    summed exactly in rationals from the double x0 and stored as two limbs.
    Returns (F, G, gamma, x0)."""
    from fractions import Fraction
    m = int(round(np.sqrt(n)))
    if m * m != n or m < 2:
        raise ValueError("the monodromy workload needs n = m^2, m >= 2")
    rng = Rng(seed * 1000003 + n)
    v = np.array([rng.unit_complex() for _ in range(m)])
    x0 = backelin_point(m, v)
    r = m - 1
    cL = np.array([[rng.unit_complex() for _ in range(n)] for _ in range(r)])
    cK = np.array([[rng.unit_complex() for _ in range(n)] for _ in range(r)])
    kK = np.array([rng.unit_complex() for _ in range(r)])
    hi, lo = np.zeros(r, dtype=np.complex128), np.zeros(r, dtype=np.complex128)
    for q in range(r):
        sr, si = Fraction(0), Fraction(0)
        for c, x in zip(cL[q], x0):
            sr -= Fraction(c.real) * Fraction(x.real) - Fraction(c.imag) * Fraction(x.imag)
            si -= Fraction(c.real) * Fraction(x.imag) + Fraction(c.imag) * Fraction(x.real)
        hr, him = float(sr), float(si)
        hi[q] = complex(hr, him)
        lo[q] = complex(float(sr - Fraction(hr)), float(si - Fraction(him)))
    f = cyclic_system(n)
    F = _with_linear_rows(f, cK, kK, np.zeros(r, dtype=np.complex128))
    g0 = f if not fixed else SystemSpec(n, n, np.zeros(n + 1, dtype=np.int32),
                                        np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32),
                                        np.zeros(0, dtype=np.int32),
                                        np.zeros(0, dtype=np.complex128))
    G = _with_linear_rows(g0, cL, hi, lo)
    return F, G, rng.unit_complex(), x0


def cyclic_monodromy_loop(seed: int, n: int) -> dict:
    """Both halves of a monodromy loop on cyclic n-roots, n = m^2 (Section
    4.2), in the fixed-row form: "out" moves the slices L (through the start
    point) to K: target [f; K], start [0; L]; "back" moves K to L: target
    [f; L], start [0; K].  A loop is one path of each, with its own constants
    (gamma = alpha out, beta back).  Returns {"out": (F, G), "back": (F, G),
    "x0": start point on L}."""
    F, G, _, x0 = cyclic_monodromy(seed, n, fixed=True)
    m = int(round(np.sqrt(n)))
    r = m - 1
    f = cyclic_system(n)
    zero = SystemSpec(n, n, np.zeros(n + 1, dtype=np.int32), np.zeros(1, dtype=np.int32),
                      np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int32),
                      np.zeros(0, dtype=np.complex128))
    # the slice rows of F (K) and of G (L): n + 1 terms each after the cyclic part
    def rows(spec, base):
        c = spec.coeff[base:].reshape(r, n + 1)
        lo = (spec.coeff_lo[base:].reshape(r, n + 1)[:, n] if spec.coeff_lo is not None
              else np.zeros(r, dtype=np.complex128))
        return c[:, :n], c[:, n], lo
    cK, kK, kKlo = rows(F, f.M)
    cL, kL, kLlo = rows(G, 0)
    return {"out": (F, G),
            "back": (_with_linear_rows(f, cL, kL, kLlo), _with_linear_rows(zero, cK, kK, kKlo)),
            "x0": x0}


def default_params(L: int, **over) -> dict:
    """Path-tracking parameters (the paper leaves them open).  Newton's
    method roughly squares the error per iteration, so from a predictor error
    e0 the residual test after m - 1 updates needs e0^(2^(m-1)) below the
    tolerance: 3 iterations reach 1e-24 (DD) from e0 ~ 1e-6, while 1e-52 (QD)
    needs a fourth.  Complex double (L = 1) stops at 1e-11, about 10^5 units
    in the last place, where the rounding of a residual evaluation stays below."""
    tol = {1: 1e-11, 2: 1e-24, 4: 1e-52}[L]
    p = dict(max_dt=0.1, min_dt={1: 1e-8, 2: 1e-12, 4: 1e-20}[L], tol_res=tol, tol_dx=tol,
             max_res=1e8, max_x=1e8, max_steps=10000, max_newton=4 if L == 4 else 3,
             pred_order=4, relax_k=1, fixed_steps=0, control=0, lin_prec=0, fixed_rows=0,
             endgame_t=0.0, cond_f32=0.0, tol_path=0.0)
    p.update(over)
    return p


@dataclass
class Workload:
    """One path-tracking job: target system f (start system g, None = total
    degree), gamma, start point x0 and tracking parameters, in L limbs."""

    name: str
    seed: int
    L: int
    f: SystemSpec
    gamma: complex
    x0: np.ndarray                  # complex, length n (doubles)
    params: dict = field(default_factory=dict)
    g: SystemSpec | None = None

    @property
    def n(self) -> int:
        return self.f.n

    def gamma_soa(self) -> np.ndarray:
        out = np.zeros((self.L, 2))
        out[0, 0], out[0, 1] = self.gamma.real, self.gamma.imag
        return out

    def x0_soa(self) -> np.ndarray:
        out = np.zeros((self.L, 2, self.n))
        out[0, 0], out[0, 1] = self.x0.real, self.x0.imag
        return out


def _limbs(prec) -> int:
    if prec in (1, "d", "D"):
        return 1
    if prec in (2, "dd", "DD"):
        return 2
    if prec in (4, "qd", "QD"):
        return 4
    raise ValueError(f"precision {prec!r}: expected dd or qd")


def dense8(seed: int = 1, prec="dd") -> Workload:
    """n=8; 8 terms per polynomial over 4 distinct variables, exponents in
    {1,2}; total-degree start system from the all-ones root; a fixed schedule
    of 100 steps with 3 Newton updates each."""
    L = _limbs(prec)
    rng = Rng(seed)
    f = dense_system(rng, 8, 8, 4, (1, 2))
    gamma = rng.unit_complex()
    return Workload("dense8_fixed100", seed, L, f, gamma, np.ones(8, dtype=np.complex128),
                    default_params(L, fixed_steps=100, max_newton=3))


def dense64(seed: int = 1, prec="dd") -> Workload:
    """n=64; 64 terms per polynomial over 16 distinct variables, exponents in
    {1,2,3}; total-degree homotopy from the all-ones root, adaptive steps."""
    L = _limbs(prec)
    rng = Rng(seed)
    f = dense_system(rng, 64, 64, 16, (1, 2, 3))
    gamma = rng.unit_complex()
    return Workload(f"dense64_{'dd' if L == 2 else 'qd'}", seed, L, f, gamma,
                    np.ones(64, dtype=np.complex128), default_params(L))


def sparse512(seed: int = 1, prec="qd") -> Workload:
    """n=512; each polynomial one linear term in x_i plus 3 monomials over 2
    other variables with exponents in {1,2}; total-degree homotopy, adaptive."""
    L = _limbs(prec)
    rng = Rng(seed)
    f = sparse_system(rng, 512)
    gamma = rng.unit_complex()
    return Workload(f"sparse512_{'dd' if L == 2 else 'qd'}", seed, L, f, gamma,
                    np.ones(512, dtype=np.complex128), default_params(L))


def sparse512_planted(seed: int = 1, prec="qd") -> tuple[Workload, np.ndarray]:
    """The sparse n = 512 recipe with a planted root x* (sparse_planted), so
    that a whole total-degree path ends at a regular root: the start root of
    x*'s path comes from tracking x* backwards.  Returns (workload, x*)."""
    L = _limbs(prec)
    rng = Rng(seed)
    f, xs = sparse_planted(rng, 512)
    gamma = rng.unit_complex()
    wl = Workload(f"sparse512_planted_{'dd' if L == 2 else 'qd'}", seed, L, f, gamma,
                  np.ones(512, dtype=np.complex128), default_params(L))
    return wl, xs


def precision128(seed: int = 1, prec="qd") -> tuple[Workload, np.ndarray]:
    """n=128; 128 terms per polynomial over 16 distinct variables, exponents in
    {1,2,3}, coefficient moduli spread log-uniformly over 12 decades within each
    polynomial and a planted root x* (planted_system).  Returns the workload (its start point is
    the all-ones root; the planted root's own start root comes from tracking x*
    backwards) and x*."""
    L = _limbs(prec)
    rng = Rng(seed)
    f, xs = planted_system(rng, 128, 128, 16, (1, 2, 3), 12.0)
    gamma = rng.unit_complex()
    wl = Workload(f"precision128_{'dd' if L == 2 else 'qd'}", seed, L, f, gamma,
                  np.ones(128, dtype=np.complex128), default_params(L))
    return wl, xs


def total_degree_start(f: SystemSpec) -> SystemSpec:
    """The total-degree start system g_i = x_i^{d_i} - 1 of f as an explicit
    system (d_i the degree of f_i), for homotopies that need it as a system
    of their own, such as tracking backwards from a root of f."""
    d = f.degrees()
    return build_system(f.N, f.n, [[(1.0, [(i, int(d[i]))]), (-1.0, [])] for i in range(f.n)])


def nearest_start_root(f: SystemSpec, x: np.ndarray) -> np.ndarray:
    """The root of x_i^{d_i} = 1 nearest to x coordinate by coordinate:
    exp(2 pi i m_i / d_i) with m_i the rounded angle, rounded to double."""
    d = f.degrees()
    m = np.round(np.angle(x) * d / (2 * np.pi)) % d
    return np.exp(2j * np.pi * m / d)


def dense64_planted(seed: int = 1, prec="dd") -> tuple[Workload, np.ndarray]:
    """The dense n = 64 recipe (64 unit-modulus terms per polynomial over 16
    distinct variables, exponents in {1, 2, 3}) with a planted root x*: each
    polynomial also gets the constant term that makes f(x*) = 0 exactly
    (planted_system with one decade of spread switched off), so the
    total-degree path that ends at x* converges.  The workload's start point is
    the all-ones root; the start root of x*'s path comes from tracking x*
    backwards.  Returns (workload, x*)."""
    L = _limbs(prec)
    rng = Rng(seed)
    f, xs = planted_system(rng, 64, 64, 16, (1, 2, 3), 0.0)
    gamma = rng.unit_complex()
    wl = Workload(f"dense64_planted_{'dd' if L == 2 else 'qd'}", seed, L, f, gamma,
                  np.ones(64, dtype=np.complex128), default_params(L))
    return wl, xs


def precision128_equations(seed: int = 1, prec="qd", decades: float = 12.0):
    """precision128's shape (n = 128, 128 terms per polynomial over 16
    variables, exponents {1, 2, 3}, planted root x*) with the coefficient
    moduli spread over `decades` decades between the equations
    (planted_system with per_equation): the Jacobian's rows differ in scale
    by up to 10^decades, which pushes its condition number up by as much.
    Returns (workload, x*)."""
    L = _limbs(prec)
    rng = Rng(seed)
    f, xs = planted_system(rng, 128, 128, 16, (1, 2, 3), decades, per_equation=True)
    gamma = rng.unit_complex()
    wl = Workload(f"precision128eq_{'dd' if L == 2 else 'qd'}", seed, L, f, gamma,
                  np.ones(128, dtype=np.complex128), default_params(L))
    return wl, xs


def random_x(rng: Rng, n: int, radius: float = 1.0) -> np.ndarray:
    """Points with coordinates of modulus radius*U[0.5, 1.5] and uniform angle."""
    return np.array([rng.unit_complex() * radius * (0.5 + rng.uniform()) for _ in range(n)])


def random_lsq(seed: int, L: int, N: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """A seeded least-squares problem in the library's layout: J [L][2][n][N]
    (column-major) and rhs [L][2][N].  Leading limbs: real and imaginary parts
    uniform in [-1, 1) (53-bit draws, so the same on every machine); limb l > 0
    is the leading limb times 2^(-60 l), an exact scaling that keeps the limbs
    non-overlapping and makes every limb of the solver's input matter."""
    rng = Rng(seed)
    lead = np.array([2.0 * rng.uniform() - 1.0 for _ in range(2 * (n + 1) * N)])
    lead = lead.reshape(n + 1, 2, N)                  # column, part, row
    J = np.zeros((L, 2, n, N))
    rhs = np.zeros((L, 2, N))
    for l in range(L):
        s = 2.0 ** (-60 * l)
        J[l] = np.transpose(lead[:n], (1, 0, 2)) * s
        rhs[l] = lead[n] * s
    return J, rhs
