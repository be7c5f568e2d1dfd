"""Global 5-point operator K (oracle; test infrastructure).

Discretisation of  lap p + kappa p = f  (Eq. 1) by central differences
(Eq. "Poisson_central", read with p_{i,j-1} for the second p_{i,j+1} the
equation prints twice) on a uniform grid with dx = dy = h:

    (p[I+1,J] + p[I-1,J] + p[I,J+1] + p[I,J-1] - 4 p[I,J]) / h^2 + kappa p[I,J] = f[I,J]

at every unknown; a neighbour that is not an unknown lies on the domain's edge
and carries zero (homogeneous Dirichlet).  For one rectangle this is the block
tridiagonal matrix of Eq. "mat_Poisson" with diagonal blocks A_y of Eq.
"submat_Dirichlet" and kappa added to the diagonal (Eq. 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import block_order_points, block_ranges


def assemble(domain: str, n: int, kappa: float = 0.0) -> sp.csr_matrix:
    """K over all unknowns of the domain, rows/columns in block order."""
    pts = block_order_points(domain, n)
    index = {p: k for k, p in enumerate(pts)}
    inv_h2 = float((n + 1) ** 2)
    rows, cols, vals = [], [], []
    for k, (I, J) in enumerate(pts):
        rows.append(k)
        cols.append(k)
        vals.append(-4.0 * inv_h2 + kappa)
        for nb in ((I + 1, J), (I - 1, J), (I, J + 1), (I, J - 1)):
            q = index.get(nb)
            if q is not None:
                rows.append(k)
                cols.append(q)
                vals.append(inv_h2)
    N = len(pts)
    return sp.csr_matrix((np.asarray(vals), (np.asarray(rows), np.asarray(cols))), shape=(N, N))


def assemble_grid(domain: str, n: int, kappa: float = 0.0) -> sp.csr_matrix:
    """The same K as `assemble`, built from a grid-shaped index map instead of a
    per-point dictionary, so that it reaches n = 512 and 1024 (1.3M and 5.2M
    unknowns) in seconds.  Every grid point (I, J) of the 3 x 3 bounding square
    gets its unknown number, or -1 where it is not an unknown; each unknown's
    row holds -4/h^2 + kappa on the diagonal and 1/h^2 for every neighbour whose
    number is not -1.  The definition is the one in `assemble`'s header; the
    tests check the two constructions give identical matrices."""
    m = n + 1
    lo = -m                                    # smallest I or J of any block's node
    grid = np.full((4 * m + 1, 4 * m + 1), -1, dtype=np.int64)   # [I - lo, J - lo]
    N = 0
    for _, i0, j0, nx, ny, off, size in block_ranges(domain, n):
        J, I = np.meshgrid(np.arange(j0, j0 + ny), np.arange(i0, i0 + nx), indexing="ij")
        grid[I - lo, J - lo] = off + np.arange(size).reshape(ny, nx)
        N = max(N, off + size)
    where = np.argwhere(grid >= 0)
    row = grid[where[:, 0], where[:, 1]]
    inv_h2 = float(m * m)
    rows, cols, vals = [row], [row], [np.full(row.size, -4.0 * inv_h2 + kappa)]
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        col = grid[where[:, 0] + di, where[:, 1] + dj]
        ok = col >= 0
        rows.append(row[ok])
        cols.append(col[ok])
        vals.append(np.full(int(ok.sum()), inv_h2))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def rectangle(nx: int, ny: int, h: float, kappa: float = 0.0) -> sp.csr_matrix:
    """5-point Dirichlet operator of one nx x ny rectangle (x fastest), Eq. "mat_Poisson"."""
    d = 1.0 / (h * h)
    ex = np.ones(nx)
    ey = np.ones(ny)
    Tx = sp.diags([ex[:-1], -2.0 * ex, ex[:-1]], [-1, 0, 1], shape=(nx, nx))
    Ty = sp.diags([ey[:-1], -2.0 * ey, ey[:-1]], [-1, 0, 1], shape=(ny, ny))
    A = d * (sp.kron(sp.identity(ny), Tx) + sp.kron(Ty, sp.identity(nx))) + kappa * sp.identity(nx * ny)
    return sp.csr_matrix(A)


def global_residual(K: sp.spmatrix, b: np.ndarray, p: np.ndarray) -> float:
    """Relative residual ||b - K p||_2 / ||b||_2."""
    return float(np.linalg.norm(b - K @ p) / np.linalg.norm(b))
