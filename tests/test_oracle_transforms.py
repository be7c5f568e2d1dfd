"""Pins for the DST-I and the closed-form eigenpairs (CPU only)."""
import numpy as np
import pytest
import scipy.fft

from oracle import transforms as T


@pytest.mark.parametrize("n", [1, 2, 7, 64, 100])
def test_Q_is_symmetric_orthogonal(n):
    Q = T.q_matrix(n)
    assert np.allclose(Q, Q.T)
    assert np.allclose(Q @ Q, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("n", [3, 16, 33])
def test_dst1_matches_library(n):
    """scipy's DST type I is 2 sum_j x_j sin(pi j k/(n+1))."""
    x = np.random.default_rng(n).standard_normal((4, n))
    assert np.allclose(T.dst1(x), scipy.fft.dst(x, type=1, axis=-1) / 2.0, atol=1e-12)


@pytest.mark.parametrize("n,dx,dy", [(9, 4.0, 4.0), (20, 100.0, 25.0)])
def test_line_eigenpairs(n, dx, dy):
    """A_y Q = Q Lambda with the closed-form eigenvalues; also equal to the
    library eigenvalues of the dense matrix."""
    A = T.line_operator(n, dx, dy)
    Q = T.q_matrix(n)
    lam = T.line_eigenvalues(n, dx, dy)
    assert np.allclose(A @ Q, Q * lam[None, :], atol=1e-10 * dx)
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(A), atol=1e-10 * dx)


def test_eigenvalue_forms_agree():
    """-4 d sin^2(theta/2) == 2 d cos(theta) - 2 d (the two textbook forms)."""
    n, h = 31, 1.0 / 32
    d = 1.0 / (h * h)
    for k in (1, 5, 31):
        a = T.rectangle_eigenvalue(k, 1, n, n, h) + 4.0 * d * np.sin(np.pi / (2 * (n + 1))) ** 2
        b = 2 * d * np.cos(k * np.pi / (n + 1)) - 2 * d
        assert abs(a - b) < 1e-9 * d
