"""Writes the stored least-squares solutions of the large MGS parity cases.

Only the oracle computes them (its textbook MGS on the augmented matrix and
back substitution: Introduction, MGS instead of LU; Section 2, N >= n least
squares).  The oracle takes minutes at these sizes, so the GPU tests read the
stored values instead of recomputing them; the inputs are regenerated from the
seed by synth.random_lsq on both sides.  Run from the repository root:

    python tests/golden/make_mgs_golden.py

Each file holds the case (L N n seed), the oracle's status, the residual norm
and the L*2*n limbs of dx (layout [L][2][n]) as exact hexadecimal doubles.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1501_06625_gb300 import synth  # noqa: E402

# (L, N, n, seed): square beyond 256 rows in DD and QD, so that every row loop
# of the solvers runs, including the one past the rows kept in registers
CASES = [(2, 288, 288, 2288), (4, 260, 260, 4260)]


def path(L: int, N: int, n: int) -> str:
    return os.path.join(HERE, f"mgs_L{L}_N{N}_n{n}.txt")


def write(L: int, N: int, n: int, seed: int) -> None:
    J, rhs = synth.random_lsq(seed, L, N, n)
    st, dx, rn = oracle.mgs_solve(J, rhs)
    with open(path(L, N, n), "w") as fh:
        fh.write(f"# oracle MGS least squares, inputs synth.random_lsq({seed}, {L}, {N}, {n})\n")
        fh.write(f"{L} {N} {n} {seed} {st}\n{float(rn).hex()}\n")
        for v in dx.reshape(-1):
            fh.write(float(v).hex() + "\n")


def read(L: int, N: int, n: int):
    """(seed, status, residual norm, dx [L][2][n]) of a stored case."""
    import numpy as np
    with open(path(L, N, n)) as fh:
        lines = [s for s in fh.read().split("\n") if s and not s.startswith("#")]
    Lr, Nr, nr, seed, st = (int(v) for v in lines[0].split())
    assert (Lr, Nr, nr) == (L, N, n)
    rn = float.fromhex(lines[1])
    dx = np.array([float.fromhex(s) for s in lines[2:]]).reshape(L, 2, n)
    return seed, st, rn, dx


if __name__ == "__main__":
    for case in CASES:
        write(*case)
        print("wrote", path(*case[:3]))
