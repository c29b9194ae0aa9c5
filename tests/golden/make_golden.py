"""Writes the oracle regression fixtures in this folder.  Calls only ``oracle/``
and the seeded input generators; run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1808_00896_gb300 import synth  # noqa: E402


def main():
    B = 4
    grid = synth.random_grid(B, seed=0x5F3F1808 + 1)
    coef = oracle.direct_forward(B, grid)  # Eq. (quadrature), summed term by term
    lmm = oracle.coef_lmm(B)
    path = os.path.join(HERE, "forward_B4_random_grid.txt")
    with open(path, "w") as f:
        f.write("# Forward SO(3) transform, B=4, of synth.random_grid(4, seed=0x5F3F1808+1),\n")
        f.write("# by the direct quadrature sum of Eq. (quadrature) (oracle.direct_forward).\n")
        f.write("# columns: l m m' re im\n")
        for (l, m, mp), c in zip(lmm, coef):
            f.write(f"{l} {m} {mp} {c.real:.17e} {c.imag:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
