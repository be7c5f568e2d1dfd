"""Unknowns of a block domain, by plain definition (oracle; test infrastructure).

A domain is a union of closed unit squares (Sec. 2.3: "concatenated"
geometry; the cross of Sec. 3).  On the uniform grid with spacing h = 1/(n+1)
the unknowns are the grid points strictly inside that union; every point on
its outer edge carries the zero Dirichlet value.  A grid point is strictly
inside iff the four grid cells that touch it all lie in the union.

The block-order listing follows the library's I/O convention (centre first,
then the arms W, E, S, N present; row-major, x fastest; the arm owns the line
it shares with the centre).  `tests/test_oracle_geometry.py` checks that this
listing is exactly the set of interior points, found independently here.
"""
from __future__ import annotations

import numpy as np

# Unit squares of each domain, as integer lower-left corners (in units of 1).
SQUARES = {
    "C": (0, 0),
    "W": (-1, 0),
    "E": (1, 0),
    "S": (0, -1),
    "N": (0, 1),
}
DOMAINS = {
    "cross": ("C", "W", "E", "S", "N"),
    "T": ("C", "W", "E", "S"),
    "L": ("C", "E", "N"),
}


def _cell_inside(domain: str, n: int, ci: int, cj: int) -> bool:
    """Is the grid cell [ci, ci+1] x [cj, cj+1] (grid units) inside the union?"""
    m = n + 1
    cx = (ci + 0.5) / m
    cy = (cj + 0.5) / m
    for b in DOMAINS[domain]:
        x0, y0 = SQUARES[b]
        if x0 < cx < x0 + 1 and y0 < cy < y0 + 1:
            return True
    return False


def interior_points(domain: str, n: int) -> set[tuple[int, int]]:
    """All integer grid points (I, J) strictly inside the domain."""
    m = n + 1
    pts = set()
    for b in DOMAINS[domain]:
        x0, y0 = SQUARES[b]
        for I in range(x0 * m, (x0 + 1) * m + 1):
            for J in range(y0 * m, (y0 + 1) * m + 1):
                if all(_cell_inside(domain, n, I + di, J + dj) for di in (-1, 0) for dj in (-1, 0)):
                    pts.add((I, J))
    return pts


def block_ranges(domain: str, n: int) -> list[tuple[str, int, int, int, int, int, int]]:
    """Per block in I/O order: (name, I_first, J_first, nx, ny, offset, size)."""
    m = n + 1
    spec = {
        "C": (1, 1, n, n),
        "W": (-m + 1, 1, n + 1, n),
        "E": (m, 1, n + 1, n),
        "S": (1, -m + 1, n, n + 1),
        "N": (1, m, n, n + 1),
    }
    out = []
    off = 0
    for b in DOMAINS[domain]:
        i0, j0, nx, ny = spec[b]
        out.append((b, i0, j0, nx, ny, off, nx * ny))
        off += nx * ny
    return out


def block_order_points(domain: str, n: int) -> list[tuple[int, int]]:
    """The unknowns listed in the library's block order."""
    pts = []
    for _, i0, j0, nx, ny, _, _ in block_ranges(domain, n):
        for j in range(ny):
            for i in range(nx):
                pts.append((i0 + i, j0 + j))
    return pts


def node_coordinates(domain: str, n: int) -> np.ndarray:
    """Physical (x, y) of the unknowns in block order, shape (N, 2)."""
    return np.asarray(block_order_points(domain, n), dtype=np.float64) / (n + 1)
