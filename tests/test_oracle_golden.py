"""The paper's worked example of reverse-mode differentiation of products of
variables (Section 3.2, Table 1), as a golden fixture for the oracle: at
dyadic points every value and partial derivative is exact, so the Jacobian
must equal the products of the other variables."""
import os
from fractions import Fraction

import numpy as np

from paper_1501_06625_gb300 import synth
from refmath import frac_vec, soa_from_complex

HERE = os.path.dirname(os.path.abspath(__file__))


def load_monomials():
    mons = []
    with open(os.path.join(HERE, "golden", "speelpenning_products.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                mons.append([int(v) for v in line.split()])
    return mons


def test_table_products(orc):
    mons = load_monomials()
    assert mons == [[0, 1, 2], [3, 4, 5], [2, 3, 4, 5], [0, 1, 3, 4, 5]]
    n = 6
    # the four products plus x_0 and x_5 alone, so that N = n as required
    mons = mons + [[0], [5]]
    spec = synth.build_system(len(mons), n, [[(1.0, [(v, 1) for v in m])] for m in mons])
    xs = np.array([2, -3, 5, 0.5, -1.5, 0.25]) + 1j * np.array([1, 0.5, -2, 1, 0, -0.75])
    for L in (2, 4):
        f = __import__("oracle").System(spec, L)
        h, J = __import__("oracle").eval_h(f, soa_from_complex(xs, L))
        xf = [complex(v) for v in xs]

        def prod(vs):
            p = (Fraction(1), Fraction(0))
            for v in vs:
                a = (Fraction(xf[v].real), Fraction(xf[v].imag))
                p = (p[0] * a[0] - p[1] * a[1], p[0] * a[1] + p[1] * a[0])
            return p

        assert frac_vec(h) == [prod(m) for m in mons]
        for j in range(n):
            col = frac_vec(J[:, :, j, :])
            want = [prod([v for v in m if v != j]) if j in m else (0, 0) for m in mons]
            assert col == want
