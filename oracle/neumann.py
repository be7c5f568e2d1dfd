"""Neumann line operator, its cosine eigenbasis and the Neumann rectangle
(oracle; test infrastructure -- only tests/, smoke() and bench.py's reference
leg use it).

Sec. 2.2, Eq. "submat_Neumann": with a zero normal derivative on the two edges
across the transform axis, the first and last rows of the line operator lose one
delta (the ghost node equals its neighbour):
    A^N = delta * tridiag(1, -2, 1) with corner entries -delta  (n x n).
Its eigenpairs (derived here; the paper's Eq. "eigenvalues_Neumann" prints
(j-1) pi/(n-1) and its Eq. "eigvector_Neumann_bar" a garbled sine form -- the
reading used is the one that diagonalises the matrix the paper prints):
    mu_k = -2 delta + 2 delta cos(k pi / n) = -4 delta sin^2(k pi/(2n)),  k = 0..n-1,
    c_k(j) = cos(k pi (j - 1/2) / n),  j = 1..n,
orthogonal with |c_0|^2 = n and |c_k|^2 = n/2 -- the DCT-II basis.  The grid in
that direction is cell-centred: x_j = (j - 1/2) h with h = 1/n.

The Neumann rectangle: n_t x n_s points, Neumann edges across t (the transform
axis), Dirichlet edges across s, 5-point stencil with the same h both ways,
kappa on the diagonal; row-major with t fastest (the library's block layout).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def neumann_line_operator(n: int, delta: float) -> np.ndarray:
    """Dense A^N of Eq. "submat_Neumann" (one direction, no kappa)."""
    A = np.diag(np.full(n, -2.0 * delta))
    A += np.diag(np.full(n - 1, delta), 1) + np.diag(np.full(n - 1, delta), -1)
    A[0, 0] += delta   # ghost node p_0 = p_1
    A[-1, -1] += delta  # ghost node p_{n+1} = p_n (both at once when n = 1)
    return A


def neumann_eigenvalues(n: int, delta: float) -> np.ndarray:
    """mu_k, k = 0..n-1."""
    k = np.arange(n)
    return -4.0 * delta * np.sin(k * np.pi / (2.0 * n)) ** 2


def dct2_matrix(n: int) -> np.ndarray:
    """C_{jk} = cos(pi k (j - 1/2) / n), j = 1..n (rows), k = 0..n-1 (columns)."""
    j = np.arange(1, n + 1) - 0.5
    k = np.arange(n)
    return np.cos(np.pi * np.outer(j, k) / n)


def dct2(x: np.ndarray) -> np.ndarray:
    """Unnormalised DCT-II along the last axis: X_k = sum_j x_j cos(pi k (j - 1/2)/n)."""
    return x @ dct2_matrix(x.shape[-1])


def idct2(X: np.ndarray) -> np.ndarray:
    """Inverse of dct2: x_j = X_0/n + (2/n) sum_{k>=1} X_k cos(pi k (j - 1/2)/n)."""
    n = X.shape[-1]
    w = np.full(n, 2.0 / n)
    w[0] = 1.0 / n
    return (X * w) @ dct2_matrix(n).T


def rectangle_neumann_t(nt: int, ns: int, h: float, kappa: float = 0.0) -> sp.csr_matrix:
    """Sparse operator of the Neumann rectangle (t fastest): Neumann across t
    (corner rows drop one delta), Dirichlet across s, kappa on the diagonal."""
    d = 1.0 / (h * h)
    At = sp.csr_matrix(neumann_line_operator(nt, d))
    As = sp.diags([np.full(ns - 1, d), np.full(ns, -2.0 * d), np.full(ns - 1, d)], [-1, 0, 1])
    return (sp.kron(sp.identity(ns), At) + sp.kron(As, sp.identity(nt)) + kappa * sp.identity(nt * ns)).tocsr()


def rectangle_neumann_mode(k: int, l: int, nt: int, ns: int) -> np.ndarray:
    """cos(k pi (j - 1/2)/nt) sin(l pi i/(ns + 1)), t fastest."""
    j = np.arange(1, nt + 1) - 0.5
    i = np.arange(1, ns + 1)
    return np.outer(np.sin(l * np.pi * i / (ns + 1)), np.cos(k * np.pi * j / nt)).ravel()


def rectangle_neumann_eigenvalue(k: int, l: int, nt: int, ns: int, h: float, kappa: float = 0.0) -> float:
    d = 1.0 / (h * h)
    return (-4.0 * d * np.sin(k * np.pi / (2.0 * nt)) ** 2
            - 4.0 * d * np.sin(l * np.pi / (2.0 * (ns + 1))) ** 2 + kappa)


def solve_neumann_rectangle(nt: int, ns: int, h: float, kappa: float, v: np.ndarray) -> np.ndarray:
    """z = A_N^{-1} v for a batch v[nvec][nt*ns] by a sparse direct solve."""
    import scipy.sparse.linalg as spla
    A = rectangle_neumann_t(nt, ns, h, kappa).tocsc()
    lu = spla.splu(A)
    v = np.atleast_2d(v)
    return np.stack([lu.solve(x) for x in v])


def manufactured(nt: int, kappa: float = 0.0):
    """p = cos(pi x) sin(pi y) on [0,1]^2 (zero x-derivative at x = 0, 1; zero at
    y = 0, 1) on the grid x_j = (j - 1/2)/nt, y_i = i/nt (ns = nt - 1, so both
    spacings are h = 1/nt); returns (h, ns, p, f) with f = lap p + kappa p."""
    h = 1.0 / nt
    ns = nt - 1
    x = (np.arange(1, nt + 1) - 0.5) * h
    y = np.arange(1, ns + 1) * h
    X, Y = np.meshgrid(x, y)  # rows: y (s), columns: x (t) -> t fastest when raveled
    p = np.cos(np.pi * X) * np.sin(np.pi * Y)
    f = (-2.0 * np.pi ** 2 + kappa) * p
    return h, ns, p.ravel(), f.ravel()
