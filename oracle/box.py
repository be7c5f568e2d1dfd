"""The 3-D extension of the fast solve on a box (oracle; test infrastructure --
only tests/, smoke() and bench.py's reference leg use it).

Sec. 2.1 (closing remark): in 3-D one more transformation turns the global
equation into independent 2-D sub-equations.  For the 7-point discretisation
of  lap p + kappa p = f  on an nx x ny x nz box with zero Dirichlet data one
step beyond every face (spacing h in all three directions, delta = 1/h^2):
    A = I_z (x) I_y (x) T_x + I_z (x) T_y (x) I_x + T_z (x) I_y (x) I_x + kappa I,
    T_m = delta tridiag(1, -2, 1) of size m,
with x fastest, then y, then z.  Its eigenvectors are the products
sin(a pi i/(nx+1)) sin(b pi j/(ny+1)) sin(c pi k/(nz+1)) and its eigenvalues
lam_a(x) + lam_b(y) + lam_c(z) + kappa with lam_a(m) = -4 delta sin^2(a pi/(2(m+1))).
A^{-1} v here is a sparse direct solve (the plain definition).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _T(m: int, d: float) -> sp.spmatrix:
    e = np.ones(m)
    return d * sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], shape=(m, m))


def box_operator(nx: int, ny: int, nz: int, h: float, kappa: float = 0.0) -> sp.csr_matrix:
    d = 1.0 / (h * h)
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    A = (sp.kron(Iz, sp.kron(Iy, _T(nx, d))) + sp.kron(Iz, sp.kron(_T(ny, d), Ix))
         + sp.kron(_T(nz, d), sp.kron(Iy, Ix)) + kappa * sp.identity(nx * ny * nz))
    return sp.csr_matrix(A)


def box_mode(a: int, b: int, c: int, nx: int, ny: int, nz: int) -> np.ndarray:
    sx = np.sin(a * np.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(b * np.pi * np.arange(1, ny + 1) / (ny + 1))
    sz = np.sin(c * np.pi * np.arange(1, nz + 1) / (nz + 1))
    return np.einsum("k,j,i->kji", sz, sy, sx).ravel()


def box_eigenvalue(a: int, b: int, c: int, nx: int, ny: int, nz: int, h: float, kappa: float = 0.0) -> float:
    d = 1.0 / (h * h)
    lam = lambda q, m: -4.0 * d * np.sin(q * np.pi / (2.0 * (m + 1))) ** 2
    return lam(a, nx) + lam(b, ny) + lam(c, nz) + kappa


def solve_box(nx: int, ny: int, nz: int, h: float, kappa: float, v: np.ndarray) -> np.ndarray:
    import scipy.sparse.linalg as spla
    lu = spla.splu(box_operator(nx, ny, nz, h, kappa).tocsc())
    return np.stack([lu.solve(x) for x in np.atleast_2d(v)])


def manufactured(n: int, kappa: float = 0.0):
    """p = sin(pi x) sin(pi y) sin(pi z) exp(0.3 x) on the unit cube, grid h = 1/(n+1),
    n^3 interior points; returns (h, p, f) with f = lap p + kappa p."""
    h = 1.0 / (n + 1)
    c = np.arange(1, n + 1) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    e = np.exp(0.3 * X)
    s = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    p = s * e
    # d2/dx2 [sin(pi x) e^{0.3x}] = e^{0.3x} [(0.09 - pi^2) sin(pi x) + 0.6 pi cos(pi x)]
    pxx = e * ((0.09 - np.pi ** 2) * np.sin(np.pi * X) + 0.6 * np.pi * np.cos(np.pi * X)) \
        * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    f = pxx - 2.0 * np.pi ** 2 * p + kappa * p
    return h, p.ravel(), f.ravel()
