"""Periodic line operator, its real eigenbasis and the periodic rectangle
(oracle; test infrastructure -- only tests/, smoke() and bench.py's reference
leg use it).

Sec. 2.2, Eq. "submat_Periodic": with periodic conditions along the transform
axis the line operator is the circulant
    A^P = delta * circ(-2, 1, 0, ..., 0, 1)   (n x n; rows 1 and n wrap around).
Eigenvalues (Eq. "eigenvalues_Periodic_corrected", here with k = j - 1):
    mu_k = -2 delta + 2 delta cos(2 pi k/n) = -4 delta sin^2(pi k/n),  k = 0..n-1,
with mu_k = mu_{n-k}.  The paper's real eigenvector matrix Q_P (Eqs.
"Q_periodic_elements"-"Periodic_mat_c_p_element", indices garbled) pairs the
frequencies k and n-k through sin(theta + pi/4) and sin(theta + 3 pi/4), i.e.
through cas(theta) = cos(theta) + sin(theta) and cas(-theta): the reading used
is the orthonormal discrete Hartley basis
    H_{jk} = cas(2 pi j k/n) / sqrt(n),   j, k = 0..n-1,
which diagonalises A^P with A^P H = H diag(mu_k).  A^{-1} does not depend on
which real eigenbasis is taken.

The periodic rectangle: n_t x n_s points, periodic along t (the transform
axis), Dirichlet across s (the edges one step beyond rows 0 and n_s-1 carry
zero), 5-point stencil with the same h both ways, kappa on the diagonal;
row-major with t fastest.  The grid along t is x_j = j h, h = 1/n_t (the period
is 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def periodic_line_operator(n: int, delta: float) -> np.ndarray:
    """Dense A^P of Eq. "submat_Periodic" (one direction, no kappa): each point
    couples to its left and right neighbour modulo n."""
    A = np.zeros((n, n))
    for j in range(n):
        A[j, j] -= 2.0 * delta
        A[j, (j + 1) % n] += delta
        A[j, (j - 1) % n] += delta
    return A


def periodic_eigenvalues(n: int, delta: float) -> np.ndarray:
    """mu_k, k = 0..n-1."""
    k = np.arange(n)
    return -4.0 * delta * np.sin(np.pi * k / n) ** 2


def hartley_matrix(n: int) -> np.ndarray:
    """H_{jk} = cas(2 pi j k/n)/sqrt(n): orthonormal, symmetric, H^2 = I."""
    jk = np.outer(np.arange(n), np.arange(n))
    a = 2.0 * np.pi * jk / n
    return (np.cos(a) + np.sin(a)) / np.sqrt(n)


def rectangle_periodic_t(nt: int, ns: int, h: float, kappa: float = 0.0) -> sp.csr_matrix:
    """Sparse operator of the periodic rectangle (t fastest)."""
    d = 1.0 / (h * h)
    At = sp.csr_matrix(periodic_line_operator(nt, d))
    As = sp.diags([np.full(ns - 1, d), np.full(ns, -2.0 * d), np.full(ns - 1, d)], [-1, 0, 1])
    return (sp.kron(sp.identity(ns), At) + sp.kron(As, sp.identity(nt)) + kappa * sp.identity(nt * ns)).tocsr()


def rectangle_periodic_mode(k: int, l: int, nt: int, ns: int) -> np.ndarray:
    """cas(2 pi k j/nt) sin(l pi i/(ns + 1)), t fastest (j = 0..nt-1, i = 1..ns)."""
    a = 2.0 * np.pi * k * np.arange(nt) / nt
    i = np.arange(1, ns + 1)
    return np.outer(np.sin(l * np.pi * i / (ns + 1)), np.cos(a) + np.sin(a)).ravel()


def rectangle_periodic_eigenvalue(k: int, l: int, nt: int, ns: int, h: float, kappa: float = 0.0) -> float:
    d = 1.0 / (h * h)
    return (-4.0 * d * np.sin(np.pi * k / nt) ** 2
            - 4.0 * d * np.sin(l * np.pi / (2.0 * (ns + 1))) ** 2 + kappa)


def solve_periodic_rectangle(nt: int, ns: int, h: float, kappa: float, v: np.ndarray) -> np.ndarray:
    """z = A_P^{-1} v for a batch v[nvec][nt*ns] by a sparse direct solve."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(rectangle_periodic_t(nt, ns, h, kappa).tocsc())
    v = np.atleast_2d(v)
    return np.stack([lu.solve(x) for x in v])


def manufactured(nt: int, kappa: float = 0.0):
    """p = (cos(2 pi x) + 0.5 sin(4 pi x)) sin(pi y) on [0,1) x [0,1], periodic in x,
    zero at y = 0 and 1, on x_j = j/nt, y_i = i/nt (ns = nt - 1, so both
    spacings are h = 1/nt); returns (h, ns, p, f) with f = lap p + kappa p."""
    h = 1.0 / nt
    ns = nt - 1
    X, Y = np.meshgrid(np.arange(nt) * h, np.arange(1, ns + 1) * h)
    g = np.cos(2 * np.pi * X) + 0.5 * np.sin(4 * np.pi * X)
    gxx = -(2 * np.pi) ** 2 * np.cos(2 * np.pi * X) - 0.5 * (4 * np.pi) ** 2 * np.sin(4 * np.pi * X)
    s = np.sin(np.pi * Y)
    p = g * s
    f = gxx * s - np.pi ** 2 * g * s + kappa * p
    return h, ns, p.ravel(), f.ravel()
