"""Independent reference arithmetic for the tests: exact rationals (fractions)
and high-precision floats (mpmath).  Converts the library's limb layout
[L][2][m] to and from exact values."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

U = 2.0 ** -53


def frac_real(limbs) -> Fraction:
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))


def frac_vec(a: np.ndarray):
    """[L][2][m] -> list of (re, im) Fractions."""
    L, _, m = a.shape
    return [(frac_real(a[:, 0, i]), frac_real(a[:, 1, i])) for i in range(m)]


def limbs_of_fraction(q: Fraction, L: int) -> list[float]:
    """Greedy split of an exact rational into L doubles (round to nearest at
    each stage); exact when q has at most ~53 L significant bits."""
    out = []
    r = q
    for _ in range(L):
        d = float(r)
        out.append(d)
        r -= Fraction(d)
    return out


def rand_limbs(rng: np.random.Generator, L: int, count: int, emin: int, emax: int) -> np.ndarray:
    """[L][count] random multi-limb reals: leading limb with a random exponent in
    [emin, emax], each next limb about 2^-53 times the one before, random sign."""
    x = np.zeros((L, count))
    lead = rng.uniform(0.5, 1.0, count) * np.exp2(rng.integers(emin, emax + 1, count)) \
        * rng.choice([-1.0, 1.0], count)
    x[0] = lead
    for l in range(1, L):
        x[l] = x[l - 1] * 2.0 ** -53 * rng.uniform(-1.0, 1.0, count)
    return x


def normalized(limbs) -> bool:
    """Each limb is at most half an ulp of the one before: fl(a + b) == a."""
    for a, b in zip(limbs[:-1], limbs[1:]):
        if a + b != a:
            return False
        if a == 0.0 and b != 0.0:
            return False
    return True


def rel_err(approx: Fraction, exact: Fraction, scale: Fraction | None = None) -> float:
    s = abs(exact) if scale is None else scale
    if s == 0:
        return 0.0 if approx == exact else math.inf
    return float(abs(approx - exact) / s)


def mp_vec(a: np.ndarray, mp):
    """[L][2][m] -> list of mpmath complex (exact conversion)."""
    L, _, m = a.shape
    out = []
    for i in range(m):
        re = mp.mpf(0)
        im = mp.mpf(0)
        for l in range(L):
            re += mp.mpf(float(a[l, 0, i]))
            im += mp.mpf(float(a[l, 1, i]))
        out.append(mp.mpc(re, im))
    return out


def soa_from_mp(vals, L: int, mp) -> np.ndarray:
    """list of mpmath complex -> [L][2][m] limbs (greedy rounding)."""
    out = np.zeros((L, 2, len(vals)))
    for i, v in enumerate(vals):
        for part, comp in ((0, v.real), (1, v.imag)):
            r = mp.mpf(comp)
            for l in range(L):
                d = float(r)
                out[l, part, i] = d
                r -= mp.mpf(d)
    return out


def soa_from_complex(z, L: int) -> np.ndarray:
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    out = np.zeros((L, 2, len(z)))
    out[0, 0], out[0, 1] = z.real, z.imag
    return out
