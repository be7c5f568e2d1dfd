"""General concatenated geometry: any edge-connected set of unit squares, with
several coupled blocks in any arrangement (oracle; test infrastructure -- only
tests/, smoke() and bench.py's CPU leg use it).

Sec. 2.3-2.4 and the remark after Alg. "fft_dd_solver": a sub-domain adjacent
to only one other is "independent" and is eliminated exactly; sub-domains
adjacent to several are "coupled" and are solved together by GMRES.  Here the
domain is a union of unit squares [i, i+1] x [j, j+1], 0 <= i, j < 8, given as a
64-bit mask (bit i + 8 j).  Grid: vertex-centred, h = 1/(n+1), m = n + 1; the
unknowns are the grid points strictly inside the union (zero Dirichlet data on
its edge).  They are partitioned into rectangular blocks:
  * every square with two or more edge neighbours is coupled and contributes its
    n x n interior points (a lone pair of squares: the first is taken as coupled);
  * every square with exactly one edge neighbour is independent and contributes
    its interior plus the grid line it shares with that neighbour -- (n+1) x n or
    n x (n+1) points, the shared line last (neighbour to the east or north) or
    first (west or south), as the arms of the cross;
  * every grid line shared by two coupled squares is a block of its own (a link,
    n points along the line), and so is every lattice vertex whose four incident
    squares are all present (a junction point).
Block order (the library's I/O convention for this geometry): the coupled set
first -- coupled squares in bit order, then the links (those across vertical
edges, ordered by (j, i) of the left square, then those across horizontal edges,
ordered by (j, i) of the lower square), then the junction points (ordered by
the vertex's (Y, X)) -- then the independent squares in bit order.  Inside a
block, x fastest.

The coupled set's own operator A_c (K restricted to it, links and junctions
included) is not one rectangle, so the paper's A_2^{-1} is generalised as the
block diagonal of the coupled set's parts: the exact inverse of each coupled
square's, each link's and each junction's own operator.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .schur import BlockSystem

E, W_, N_, S_ = (1, 0), (-1, 0), (0, 1), (0, -1)


def squares(mask: int) -> list[tuple[int, int]]:
    """Lower-left corners (i, j) of the squares, in bit order (bit i + 8 j)."""
    return [(b % 8, b // 8) for b in range(64) if (mask >> b) & 1]


def neighbours(mask: int, sq: tuple[int, int]) -> list[tuple[int, int]]:
    """Directions (di, dj) to the edge neighbours of square sq that are present."""
    have = set(squares(mask))
    return [d for d in (E, W_, N_, S_) if (sq[0] + d[0], sq[1] + d[1]) in have]


def connected(mask: int) -> bool:
    sq = squares(mask)
    if not sq:
        return False
    seen, todo = {sq[0]}, [sq[0]]
    while todo:
        c = todo.pop()
        for d in neighbours(mask, c):
            nb = (c[0] + d[0], c[1] + d[1])
            if nb not in seen:
                seen.add(nb)
                todo.append(nb)
    return len(seen) == len(sq)


def classify(mask: int):
    """(coupled squares, {independent square: direction to its neighbour}), both in
    bit order.  Squares with >= 2 neighbours are coupled; with exactly 1,
    independent; if that leaves no coupled square (two squares), the first is
    coupled."""
    sq = squares(mask)
    coupled = [s for s in sq if len(neighbours(mask, s)) >= 2]
    if not coupled:
        coupled = [sq[0]]
    indep = {s: neighbours(mask, s)[0] for s in sq if s not in coupled}
    return coupled, indep


def links(mask: int):
    """Grid lines shared by two coupled squares: ('V', i, j) for the vertical edge
    x = i + 1 between (i, j) and (i + 1, j), then ('H', i, j) for the horizontal
    edge y = j + 1 between (i, j) and (i, j + 1), each kind ordered by (j, i)."""
    coupled = set(classify(mask)[0])
    out = []
    for kind, d in (("V", E), ("H", N_)):
        for j in range(8):
            for i in range(8):
                if (i, j) in coupled and (i + d[0], j + d[1]) in coupled:
                    out.append((kind, i, j))
    return out


def junctions(mask: int):
    """Lattice vertices (X, Y) whose four incident squares are all present, ordered by (Y, X)."""
    have = set(squares(mask))
    return [(X, Y) for Y in range(1, 8) for X in range(1, 8)
            if {(X - 1, Y - 1), (X, Y - 1), (X - 1, Y), (X, Y)} <= have]


def interior_points(mask: int, n: int) -> set:
    """Grid points (I, J) (units of h) strictly inside the union: all four grid
    cells around the point lie in some square (found from the squares alone)."""
    m = n + 1
    have = set(squares(mask))

    def cell_in(ci, cj):  # the cell [ci, ci+1] x [cj, cj+1] of the grid
        return (ci // m, cj // m) in have

    pts = set()
    for i, j in have:
        for I in range(i * m, (i + 1) * m + 1):
            for J in range(j * m, (j + 1) * m + 1):
                if all(cell_in(I + a, J + b) for a in (-1, 0) for b in (-1, 0)):
                    pts.add((I, J))
    return pts


def block_ranges(mask: int, n: int) -> list:
    """(name, I_first, J_first, nx, ny, offset, size) per block, in block order."""
    m = n + 1
    coupled, indep = classify(mask)
    spec = [(f"Q{i}_{j}", i * m + 1, j * m + 1, n, n) for i, j in coupled]
    for kind, i, j in links(mask):
        if kind == "V":
            spec.append((f"V{i}_{j}", (i + 1) * m, j * m + 1, 1, n))
        else:
            spec.append((f"H{i}_{j}", i * m + 1, (j + 1) * m, n, 1))
    spec += [(f"P{X}_{Y}", X * m, Y * m, 1, 1) for X, Y in junctions(mask)]
    for (i, j), d in indep.items():
        if d == E:
            spec.append((f"A{i}_{j}", i * m + 1, j * m + 1, m, n))
        elif d == W_:
            spec.append((f"A{i}_{j}", i * m, j * m + 1, m, n))
        elif d == N_:
            spec.append((f"A{i}_{j}", i * m + 1, j * m + 1, n, m))
        else:
            spec.append((f"A{i}_{j}", i * m + 1, j * m, n, m))
    out, off = [], 0
    for name, i0, j0, nx, ny in spec:
        out.append((name, i0, j0, nx, ny, off, nx * ny))
        off += nx * ny
    return out


def block_order_points(mask: int, n: int) -> list:
    pts = []
    for _, i0, j0, nx, ny, _, _ in block_ranges(mask, n):
        for j in range(ny):
            for i in range(nx):
                pts.append((i0 + i, j0 + j))
    return pts


def coupled_size(mask: int, n: int) -> int:
    """Unknowns of the coupled set (the Krylov vector's length)."""
    return sum(b[6] for b in block_ranges(mask, n) if b[0][0] in "QVHP")


def node_coordinates(mask: int, n: int) -> np.ndarray:
    return np.asarray(block_order_points(mask, n), dtype=np.float64) / (n + 1)


def assemble(mask: int, n: int, kappa: float = 0.0) -> sp.csr_matrix:
    """The global 5-point K of  lap p + kappa p = f  (Eq. 1, Eq. "Poisson_central")
    over the unknowns in block order; a neighbour that is not an unknown lies on
    the edge of the union and carries zero."""
    pts = block_order_points(mask, n)
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


def assemble_grid(mask: int, n: int, kappa: float = 0.0) -> sp.csr_matrix:
    """The same K from a grid-shaped index map (for n up to 512); the tests check
    it equals `assemble` entry for entry."""
    m = n + 1
    grid = np.full((8 * m + 1, 8 * m + 1), -1, dtype=np.int64)  # [I, J]
    for _, i0, j0, nx, ny, off, size in block_ranges(mask, n):
        J, I = np.meshgrid(np.arange(j0, j0 + ny), np.arange(i0, i0 + nx), indexing="ij")
        grid[I, J] = off + np.arange(size).reshape(ny, nx)
    N = sum(b[6] for b in block_ranges(mask, n))
    where = np.argwhere(grid >= 0)
    row = grid[where[:, 0], where[:, 1]]
    d = float(m * m)
    rows, cols, vals = [row], [row], [np.full(row.size, -4.0 * d + kappa)]
    for di, dj in (E, W_, N_, S_):
        I, J = where[:, 0] + di, where[:, 1] + dj
        ok = (I >= 0) & (J >= 0) & (I < grid.shape[0]) & (J < grid.shape[1])
        col = np.full(row.size, -1, dtype=np.int64)
        col[ok] = grid[I[ok], J[ok]]
        ok = col >= 0
        rows.append(row[ok])
        cols.append(col[ok])
        vals.append(np.full(int(ok.sum()), d))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def block_system(mask: int, n: int, K: sp.spmatrix) -> tuple[BlockSystem, list]:
    """The Schur structure of Sec. 2.3 with the coupled set as the 'centre'
    vector: (BlockSystem, index arrays of the coupled set's parts -- each coupled
    square, link and junction -- for the block-diagonal preconditioner)."""
    br = block_ranges(mask, n)
    nc = coupled_size(mask, n)
    blocks = [("C", 0, 0, 0, 0, 0, nc)] + [b for b in br if b[0][0] == "A"]
    parts = [np.arange(b[5], b[5] + b[6]) for b in br if b[0][0] in "QVHP"]
    return BlockSystem(K, "lattice", n, blocks=blocks), parts
