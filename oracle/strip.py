"""A domain with several coupled blocks: a chain of K crosses (oracle; test
infrastructure -- only tests/, smoke() and bench.py's reference leg use it).

Sec. 2.3-2.4: a block adjacent to one other block is "independent" and is
eliminated exactly; blocks adjacent to several blocks are "coupled" and are
solved together by GMRES.  The chain: 2K - 1 unit squares side by side along x
([q, q+1] x [0, 1], q = 0..2K-2) -- the centres C_i at q = 2(i-1) and the links
between them at odd q -- an arm W left of the first square, an arm E right of
the last, and arms S_i below and N_i above every centre C_i.  Every square of
the row touches two or more blocks (coupled); the 2K + 2 arms touch one
(independent) and no two arms touch along an edge.  K = 1 is the cross.

Grid: vertex-centred, h = 1/(n+1); the unknowns are the grid points strictly
inside the union (zero Dirichlet data on its edge), found here from the squares
alone.  Block order (the library's I/O convention for chains):
  * the coupled row as one rectangle: x = h .. (2K-1) - h, y = h .. 1 - h, i.e.
    nx_c = (2K-1)(n+1) - 1 columns by n rows, x fastest (each square owns the line
    it shares with the next one);
  * W and E, (n+1) x n each, owning the line they share with the row;
  * S_1..S_K, then N_1..N_K, n x (n+1) each, owning their shared line.
The preconditioner of the coupled set (the paper's A_2^{-1} generalised to
several coupled blocks) is block-diagonal: the exact inverse of each square's
own operator on its columns, x in (q, q+1] for q < 2K-2 (n+1 columns) and the
last square's n columns.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def squares(K: int) -> dict:
    """Lower-left corners of the unit squares of the chain, by block name."""
    sq = {f"R{q}": (q, 0) for q in range(2 * K - 1)}
    sq["W"] = (-1, 0)
    sq["E"] = (2 * K - 1, 0)
    for i in range(1, K + 1):
        sq[f"S{i}"] = (2 * (i - 1), -1)
        sq[f"N{i}"] = (2 * (i - 1), 1)
    return sq


def interior_points(K: int, n: int) -> set:
    """Grid points (I, J) (units of h) strictly inside the union: all four grid
    cells around the point lie in some square."""
    m = n + 1
    sq = list(squares(K).values())

    def cell_in(ci, cj):
        cx, cy = (ci + 0.5) / m, (cj + 0.5) / m
        return any(x0 < cx < x0 + 1 and y0 < cy < y0 + 1 for x0, y0 in sq)

    pts = set()
    for x0, y0 in sq:
        for I in range(x0 * m, (x0 + 1) * m + 1):
            for J in range(y0 * m, (y0 + 1) * m + 1):
                if all(cell_in(I + a, J + b) for a in (-1, 0) for b in (-1, 0)):
                    pts.add((I, J))
    return pts


def block_ranges(K: int, n: int) -> list:
    """(name, I_first, J_first, nx, ny, offset, size) per block in I/O order."""
    m = n + 1
    q = 2 * K - 1
    spec = [("C", 1, 1, q * m - 1, n), ("W", -m + 1, 1, m, n), ("E", q * m, 1, m, n)]
    spec += [(f"S{i}", 2 * (i - 1) * m + 1, -m + 1, n, m) for i in range(1, K + 1)]
    spec += [(f"N{i}", 2 * (i - 1) * m + 1, m, n, m) for i in range(1, K + 1)]
    out, off = [], 0
    for b, i0, j0, nx, ny in spec:
        out.append((b, i0, j0, nx, ny, off, nx * ny))
        off += nx * ny
    return out


def block_order_points(K: int, n: int) -> list:
    pts = []
    for _, i0, j0, nx, ny, _, _ in block_ranges(K, n):
        for j in range(ny):
            for i in range(nx):
                pts.append((i0 + i, j0 + j))
    return pts


def assemble(K: int, n: int, kappa: float = 0.0) -> sp.csr_matrix:
    """The global 5-point K over the strip's unknowns in block order; a neighbour
    that is not an unknown lies on the edge and carries zero."""
    pts = block_order_points(K, n)
    index = {p: k for k, p in enumerate(pts)}
    d = float((n + 1) ** 2)
    rows, cols, vals = [], [], []
    for k, (I, J) in enumerate(pts):
        rows.append(k)
        cols.append(k)
        vals.append(-4.0 * d + kappa)
        for nb in ((I + 1, J), (I - 1, J), (I, J + 1), (I, J - 1)):
            q = index.get(nb)
            if q is not None:
                rows.append(k)
                cols.append(q)
                vals.append(d)
    N = len(pts)
    return sp.csr_matrix((np.asarray(vals), (np.asarray(rows), np.asarray(cols))), shape=(N, N))


def centre_block_columns(K: int, n: int) -> list:
    """Column ranges (first, count) of the 2K - 1 coupled squares inside the row."""
    m = n + 1
    q = 2 * K - 1
    return [(s * m, m if s < q - 1 else n) for s in range(q)]


def coordinates(K: int, n: int) -> np.ndarray:
    return np.asarray(block_order_points(K, n), dtype=np.float64) / (n + 1)
