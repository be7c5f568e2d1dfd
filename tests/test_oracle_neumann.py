"""Pins of the Neumann oracle (Sec. 2.2, Eq. "submat_Neumann"): eigenpairs in
closed form, the transform against a library DCT, an independently built dense
stencil, second-order convergence on a manufactured solution, and the rectangle
solve by an independent route (library DCT-II plus banded solves)."""
import numpy as np
import pytest

from oracle import neumann as N


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_cosine_basis_diagonalises_the_neumann_line_operator(n):
    delta = 7.0
    A = N.neumann_line_operator(n, delta)
    C = N.dct2_matrix(n)
    mu = N.neumann_eigenvalues(n, delta)
    assert np.allclose(A @ C, C * mu, atol=1e-12 * delta)
    # orthogonal columns, |c_0|^2 = n, |c_k|^2 = n/2
    G = C.T @ C
    want = np.full(n, n / 2.0)
    want[0] = n
    assert np.allclose(G, np.diag(want), atol=1e-12 * n)
    # the spectrum of the matrix, independently
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(mu), atol=1e-12 * delta)


def test_dct2_matches_scipy_and_inverts():
    fft = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 24))
    X = N.dct2(x)
    assert np.allclose(X, fft.dct(x, type=2, axis=-1) / 2.0, atol=1e-12)
    assert np.allclose(N.idct2(X), x, atol=1e-12)


def _dense_stencil(nt, ns, h, kappa):
    """Neumann rectangle built point by point from the 5-point stencil with ghost
    nodes p_0 = p_1 and p_{nt+1} = p_nt along t, zeros outside along s."""
    d = 1.0 / h ** 2
    A = np.zeros((nt * ns, nt * ns))
    for i in range(ns):
        for j in range(nt):
            r = i * nt + j
            A[r, r] += -4.0 * d + kappa
            for dj in (-1, 1):
                jj = j + dj
                jj = j if jj < 0 or jj >= nt else jj  # ghost = mirror of the boundary point
                A[r, i * nt + jj] += d
            for di in (-1, 1):
                ii = i + di
                if 0 <= ii < ns:
                    A[r, ii * nt + j] += d
    return A


@pytest.mark.parametrize("nt,ns,kappa", [(2, 3, 0.0), (4, 4, -3.0), (6, 5, -10.0)])
def test_sparse_operator_equals_point_stencil(nt, ns, kappa):
    h = 0.25
    assert np.allclose(N.rectangle_neumann_t(nt, ns, h, kappa).toarray(), _dense_stencil(nt, ns, h, kappa))


@pytest.mark.parametrize("k,l", [(0, 1), (3, 2), (7, 5)])
def test_rectangle_modes_are_eigenvectors(k, l):
    nt, ns, h, kappa = 8, 6, 1.0 / 8, -10.0
    A = N.rectangle_neumann_t(nt, ns, h, kappa)
    q = N.rectangle_neumann_mode(k, l, nt, ns)
    lam = N.rectangle_neumann_eigenvalue(k, l, nt, ns, h, kappa)
    assert np.allclose(A @ q, lam * q, atol=1e-10 * abs(lam))


def test_solve_is_the_dense_inverse_on_small_rectangles():
    nt, ns, h, kappa = 6, 5, 0.2, -3.0
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2, nt * ns))
    z = N.solve_neumann_rectangle(nt, ns, h, kappa, v)
    assert np.allclose(z, np.linalg.solve(_dense_stencil(nt, ns, h, kappa), v.T).T, atol=1e-12)


def test_second_order_on_the_manufactured_solution():
    errs = []
    for nt in (16, 32, 64):
        h, ns, p, f = N.manufactured(nt)
        z = N.solve_neumann_rectangle(nt, ns, h, 0.0, f[None, :])[0]
        errs.append(np.max(np.abs(z - p)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_direct_solve_equals_dct_banded_solve():
    """An independent route: scipy's orthonormal DCT-II along t, one banded
    (tridiagonal) solve per cosine mode along s, inverse DCT-II -- equal to the
    sparse LU solve of the Neumann rectangle."""
    from scipy.fft import dct, idct
    from scipy.linalg import solve_banded
    nt, ns, h, kappa = 11, 8, 1.0 / 11, -3.0
    d = 1.0 / h ** 2
    v = np.random.default_rng(6).standard_normal((ns, nt))
    V = dct(v, type=2, norm="ortho", axis=1)
    Z = np.empty_like(V)
    for k in range(nt):
        ab = np.zeros((3, ns))
        ab[0, 1:] = d
        ab[1, :] = -2 * d - 4 * d * np.sin(np.pi * k / (2 * nt)) ** 2 + kappa
        ab[2, :-1] = d
        Z[:, k] = solve_banded((1, 1), ab, V[:, k])
    z = idct(Z, type=2, norm="ortho", axis=1)
    want = N.solve_neumann_rectangle(nt, ns, h, kappa, v.ravel()[None, :])[0]
    assert np.allclose(z.ravel(), want, rtol=1e-11, atol=1e-13)
