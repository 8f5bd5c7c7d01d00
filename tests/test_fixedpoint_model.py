"""A CPU model of the straight-line round-back of the fixed-point sums
(exsum.cuh: fix_round2 for 128-bit, fix_round4 for 256-bit accumulators),
step for step as the device code does it, checked against exact rounding in
rationals: each limb must be the double nearest to what the previous limbs
leave (round to nearest, ties to even).  The device code itself is checked on
the GPU (tests/test_gpu_exsum.py, tests/test_gpu_fixedpoint.py); this model
pins the algorithm -- normalisation, the rounding bit and sticky bits, the
carry when rounding up overflows the significand, the signed remainder --
on many more values, including forced ties and near-ties, than a GPU test
can afford to check in rationals."""
import math
import random
from fractions import Fraction

M64 = (1 << 64) - 1
M256 = (1 << 256) - 1


def _make(m, E):
    """The double m 2^E (m with its top bit at bit 52), zero below the normal
    range, infinity above it (fix_make_double)."""
    ex = E + 52
    if ex > 1023:
        return math.inf
    if ex < -1022:
        return 0.0
    return math.ldexp(m, E)


def _norm128(h, l):
    lz = (64 - h.bit_length()) if h else 64 + (64 - l.bit_length())
    n = ((h << 64) | l) << lz & ((1 << 128) - 1)
    n1, n0 = n >> 64, n & M64
    m = n1 >> 11
    r = n1 & 0x7ff
    up = bool(r & 0x400) and bool((r & 0x3ff) or n0 or (m & 1))
    return lz, m, up, r, n0


def round2(acc, base):
    """Model of fix_round2: acc a 128-bit two's-complement integer."""
    h, l = acc >> 64, acc & M64
    neg = h >> 63
    if neg:
        l = (~l + 1) & M64
        h = (~h + (1 if l == 0 else 0)) & M64
    if h | l == 0:
        return 0.0, 0.0
    lz, m, up, r, n0 = _norm128(h, l)
    e = 127 - lz - 52 + base
    mu = m + up
    v0 = _make(1 << 52, e + 1) if mu >> 53 else _make(mu, e)
    R1, R0 = r - (0x800 if up else 0), n0
    rneg = R1 < 0
    if rneg:
        R0 = (~R0 + 1) & M64
        R1 = ~R1 + (1 if R0 == 0 else 0)
    v1 = 0.0
    if R1 or R0:
        lz2, m2, up2, _, _ = _norm128(R1 & M64, R0)
        e2 = 127 - lz2 - 52 + base - lz
        mu2 = m2 + up2
        v1 = _make(1 << 52, e2 + 1) if mu2 >> 53 else _make(mu2, e2)
        if rneg:
            v1 = -v1
    return (-v0, -v1) if neg else (v0, v1)


def round4(acc, base):
    """Model of fix_round4: acc a 256-bit two's-complement integer."""
    a = acc & M256
    v = [0.0] * 4
    for l in range(4):
        neg = a >> 255
        mag = ((-a) & M256) if neg else a
        if mag == 0:
            break
        lz = 256 - mag.bit_length()
        n = (mag << lz) & M256
        w3 = n >> 192
        m, r = w3 >> 11, w3 & 0x7ff
        sticky = (r & 0x3ff) or (n & ((1 << 192) - 1))
        up = bool(r & 0x400) and bool(sticky or (m & 1))
        e = base - lz + 203
        mu = m + up
        d = _make(1 << 52, e + 1) if mu >> 53 else _make(mu, e)
        v[l] = -d if neg else d
        top = (r - (0x800 if up else 0)) & M64
        n = (top << 192) | (n & ((1 << 192) - 1))
        a = ((-n) & M256) if neg else n
        base -= lz
    return v


def _exact_limbs(x: Fraction, L):
    out = []
    for _ in range(L):
        d = float(x)                                 # correctly rounded, ties to even
        out.append(d)
        x -= Fraction(d)
    return out


def _draw(rng, widths, width_total):
    bits = rng.choice(widths)
    mag = rng.getrandbits(bits) | (1 << (bits - 1))
    if rng.random() < 0.3:                           # ties and near-ties below the 53 bits
        k = rng.randint(1, bits - 1)
        mag = (mag >> k << k) | rng.choice([0, 1 << (k - 1), (1 << (k - 1)) - 1])
    if mag >= 1 << (width_total - 2):
        mag >>= 1
    return -mag if rng.random() < 0.5 else mag


def test_round2_model_matches_exact_rounding():
    rng = random.Random(1)
    for _ in range(20000):
        val = _draw(rng, [20, 53, 54, 60, 75, 100, 120, 126], 128)
        base = rng.randint(-200, 100)
        got = round2(val & ((1 << 128) - 1), base)
        assert list(got) == _exact_limbs(Fraction(val) * Fraction(2) ** base, 2), (val, base)


def test_round4_model_matches_exact_rounding():
    rng = random.Random(3)
    for _ in range(20000):
        val = _draw(rng, [30, 53, 106, 160, 200, 230, 253], 256)
        base = rng.randint(-600, 100)
        got = round4(val & M256, base)
        assert got == _exact_limbs(Fraction(val) * Fraction(2) ** base, 4), (val, base)


def test_models_on_edges():
    # zero, one bit, all ones below the top, the most negative representable sums
    assert round2(0, 0) == (0.0, 0.0) and round4(0, 0) == [0.0] * 4
    assert round2(1, -10) == (2.0 ** -10, 0.0)
    x = (1 << 126) - 1                               # rounds up and carries into a new bit
    assert list(round2(x, 0)) == _exact_limbs(Fraction(x), 2)
    y = (1 << 254) - 1
    assert round4(y, 0) == _exact_limbs(Fraction(y), 4)
    assert round4((-y) & M256, -7) == _exact_limbs(Fraction(-y) / 128, 4)
