"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
Each file holds the oracle's direct solution p = K^{-1} f (Eq. "block_global"
solved exactly) for a small seeded workload, one value per line in the
library's block order, printed with 17 significant digits.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import direct, operator  # noqa: E402

CASES = [
    # (file, domain, n, kappa, kind, seed)
    ("cross_n8_k0_manufactured.txt", "cross", 8, 0.0, "manufactured", 0),
    ("T_n9_km10_fourier_s3.txt", "T", 9, -10.0, "fourier", 3),
    ("L_n6_k0_fourier_s1.txt", "L", 6, 0.0, "fourier", 1),
]


def expected(domain, n, kappa, kind, seed):
    f = W.rhs_batch(domain, n, [seed], kind=kind, kappa=kappa)[0]
    return f, direct.solve(operator.assemble(domain, n, kappa), f)


def main():
    for fname, domain, n, kappa, kind, seed in CASES:
        _, p = expected(domain, n, kappa, kind, seed)
        with open(os.path.join(HERE, fname), "w") as fh:
            fh.write(f"# oracle p = K^-1 f: domain={domain} n={n} kappa={kappa} kind={kind} seed={seed}\n")
            for v in p:
                fh.write(f"{v:.17g}\n")


if __name__ == "__main__":
    main()
