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


# The widening geometries: (file, geometry, n, kappa, extra) -- the Neumann-sided
# cross with the validation source (Sec. 3.1), a chain of crosses (`extra` = K)
# with the fourier workload of seed 2.
EXTRA_CASES = [
    ("ncross_n8_km10_validation.txt", "ncross", 8, -10.0, 0),
    ("chain_K2_n5_k0_fourier_s2.txt", "chain", 5, 0.0, 2),
]


def expected(domain, n, kappa, kind, seed):
    f = W.rhs_batch(domain, n, [seed], kind=kind, kappa=kappa)[0]
    return f, direct.solve(operator.assemble(domain, n, kappa), f)


def expected_extra(geometry, n, kappa, extra):
    if geometry == "ncross":
        from oracle import neumann_cross
        f = W.ncross_validation_rhs(n, kappa)
        return f, direct.solve(neumann_cross.assemble(n, kappa), f)
    from oracle import strip
    f = W.strip_fourier_rhs(extra, n, 2)
    return f, direct.solve(strip.assemble(extra, n, kappa), f)


def write(fname, header, p):
    with open(os.path.join(HERE, fname), "w") as fh:
        fh.write(f"# oracle p = K^-1 f: {header}\n")
        for v in p:
            fh.write(f"{v:.17g}\n")


def main():
    for fname, domain, n, kappa, kind, seed in CASES:
        _, p = expected(domain, n, kappa, kind, seed)
        write(fname, f"domain={domain} n={n} kappa={kappa} kind={kind} seed={seed}", p)
    for fname, geometry, n, kappa, extra in EXTRA_CASES:
        _, p = expected_extra(geometry, n, kappa, extra)
        write(fname, f"geometry={geometry} n={n} kappa={kappa} extra={extra}", p)


if __name__ == "__main__":
    main()
