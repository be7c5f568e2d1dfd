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

from .geometry import block_order_points


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
