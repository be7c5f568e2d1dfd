"""DST-I and the closed-form eigenpairs of A_y (oracle; test infrastructure).

Sec. 2.1: the Dirichlet line operator A_y^D = tridiag(dy, -2(dx+dy), dy)
(Eq. "submat_Dirichlet") has eigenvalues
    lambda_k = -2(dx+dy) + 2 dy cos(k pi/(n+1)),  k = 1..n   (Eq. "Poisson_spectral_eigen")
and orthonormal eigenvectors
    q_{j,k} = sqrt(2/(n+1)) sin(j k pi/(n+1))                (Eq. "eigvector_Diri").
The paper's fast route to Q p (Eq. "Dirichlet_mat_decomp") is garbled in its
sizes and scale; the reading used throughout is: DST-I_n(x)_k =
sum_{j=1..n} x_j sin(pi j k/(n+1)), Q = sqrt(2/(n+1)) DST-I, Q Q = I.
Here the transform is the plain dense matrix, which is what the definition says.
"""
from __future__ import annotations

import numpy as np


def dst1_matrix(n: int) -> np.ndarray:
    """S_{jk} = sin(pi j k / (n+1)), j, k = 1..n (unnormalised DST-I)."""
    j = np.arange(1, n + 1)
    return np.sin(np.pi * np.outer(j, j) / (n + 1))


def q_matrix(n: int) -> np.ndarray:
    """Orthonormal eigenvector matrix Q_D of Eq. "eigvector_Diri"."""
    return np.sqrt(2.0 / (n + 1)) * dst1_matrix(n)


def dst1(x: np.ndarray) -> np.ndarray:
    """Unnormalised DST-I along the last axis."""
    return x @ dst1_matrix(x.shape[-1])


def line_eigenvalues(n: int, dx: float, dy: float) -> np.ndarray:
    """lambda_k of A_y^D, k = 1..n (Eq. "Poisson_spectral_eigen")."""
    k = np.arange(1, n + 1)
    return -2.0 * (dx + dy) + 2.0 * dy * np.cos(k * np.pi / (n + 1))


def line_operator(n: int, dx: float, dy: float) -> np.ndarray:
    """Dense A_y^D of Eq. "submat_Dirichlet"."""
    A = np.diag(np.full(n, -2.0 * (dx + dy)))
    A += np.diag(np.full(n - 1, dy), 1) + np.diag(np.full(n - 1, dy), -1)
    return A


def rectangle_eigenvalue(k: int, l: int, nx: int, ny: int, h: float, kappa: float = 0.0) -> float:
    """Eigenvalue of the nx x ny 5-point Dirichlet operator for the mode
    sin(k pi i/(nx+1)) sin(l pi j/(ny+1)): the sum of the two line eigenvalues
    (each 1-D second difference contributes -(4/h^2) sin^2(theta/2)) plus kappa."""
    d = 1.0 / (h * h)
    return (-4.0 * d * np.sin(k * np.pi / (2 * (nx + 1))) ** 2
            - 4.0 * d * np.sin(l * np.pi / (2 * (ny + 1))) ** 2 + kappa)


def rectangle_mode(k: int, l: int, nx: int, ny: int) -> np.ndarray:
    """The mode sin(k pi i/(nx+1)) sin(l pi j/(ny+1)) on the grid, row-major (x fastest)."""
    i = np.arange(1, nx + 1)
    j = np.arange(1, ny + 1)
    return np.outer(np.sin(l * np.pi * j / (ny + 1)), np.sin(k * np.pi * i / (nx + 1))).ravel()
