"""Pins of the periodic oracle (Sec. 2.2, Eqs. "submat_Periodic",
"eigenvalues_Periodic_corrected", the real eigenbasis read as the discrete
Hartley basis) against facts independent of it: a stencil applied point by
point, numpy's FFT, symmetric eigenvalues, the circulant's translation
invariance, closed-form rectangle modes and second-order convergence."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import periodic as P


@pytest.mark.parametrize("n", [2, 3, 8, 15])
def test_line_operator_is_the_wrapped_stencil(n):
    d = 3.0
    A = P.periodic_line_operator(n, d)
    x = np.random.default_rng(n).standard_normal(n)
    want = d * (np.roll(x, 1) + np.roll(x, -1) - 2 * x)
    assert np.allclose(A @ x, want)
    # translation invariance: A commutes with the cyclic shift
    S = np.roll(np.eye(n), 1, axis=0)
    assert np.allclose(A @ S, S @ A)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_eigenpairs(n):
    d = 2.0
    A = P.periodic_line_operator(n, d)
    mu = P.periodic_eigenvalues(n, d)
    H = P.hartley_matrix(n)
    assert np.allclose(H @ H.T, np.eye(n), atol=1e-13)
    assert np.allclose(A @ H, H * mu, atol=1e-12)
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(mu), atol=1e-12)
    # the eigenvalues are the DFT of the stencil's first column (numpy's FFT)
    assert np.allclose(np.fft.fft(A[:, 0]).real, mu, atol=1e-12)


def test_hartley_is_the_fft_combination():
    """H x = (Re F x - Im F x)/sqrt(n) with F numpy's (e^{-2 pi i jk/n}) FFT."""
    n = 10
    x = np.random.default_rng(1).standard_normal(n)
    F = np.fft.fft(x)
    assert np.allclose(P.hartley_matrix(n) @ x, (F.real - F.imag) / np.sqrt(n))


@pytest.mark.parametrize("nt,ns", [(4, 3), (9, 5), (16, 16)])
def test_rectangle_modes(nt, ns):
    h, kappa = 1.0 / nt, -7.0
    A = P.rectangle_periodic_t(nt, ns, h, kappa)
    for k, l in [(0, 1), (1, ns), (nt // 2, 2), (nt - 1, 1)]:
        q = P.rectangle_periodic_mode(k, l, nt, ns)
        lam = P.rectangle_periodic_eigenvalue(k, l, nt, ns, h, kappa)
        assert np.allclose(A @ q, lam * q, atol=1e-9 * abs(lam))


def test_direct_solve_against_dense():
    nt, ns, h, kappa = 6, 5, 0.2, -1.0
    v = np.random.default_rng(3).standard_normal((2, nt * ns))
    z = P.solve_periodic_rectangle(nt, ns, h, kappa, v)
    Ad = P.rectangle_periodic_t(nt, ns, h, kappa).toarray()
    assert np.allclose(Ad @ z.T, v.T)
    assert np.allclose(np.linalg.solve(Ad, v.T).T, z)


def test_second_order_convergence():
    errs = []
    for nt in (16, 32, 64):
        h, ns, p, f = P.manufactured(nt)
        z = spla.spsolve(P.rectangle_periodic_t(nt, ns, h).tocsc(), f)
        errs.append(np.abs(z - p).max())
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2, errs


def test_direct_solve_equals_fft_banded_solve():
    """An independent route: numpy's FFT along t, one banded (tridiagonal) solve per
    Fourier mode along s with scipy, inverse FFT -- equal to the sparse LU solve."""
    from scipy.linalg import solve_banded
    nt, ns, h, kappa = 12, 9, 0.1, -2.0
    d = 1.0 / h ** 2
    v = np.random.default_rng(5).standard_normal((ns, nt))
    V = np.fft.fft(v, axis=1)
    Z = np.empty_like(V)
    for k in range(nt):
        diag = -2 * d - 4 * d * np.sin(np.pi * k / nt) ** 2 + kappa
        ab = np.zeros((3, ns), dtype=complex)
        ab[0, 1:] = d
        ab[1, :] = diag
        ab[2, :-1] = d
        Z[:, k] = solve_banded((1, 1), ab, V[:, k])
    z = np.fft.ifft(Z, axis=1).real
    want = P.solve_periodic_rectangle(nt, ns, h, kappa, v.ravel()[None, :])[0]
    assert np.allclose(z.ravel(), want, rtol=1e-11, atol=1e-13)
