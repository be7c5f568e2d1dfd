"""Pins of the 3-D box oracle (the 3-D extension named after Sec. 2.1): the
Kronecker assembly against a point-by-point 7-point stencil, closed-form
eigenmodes, symmetry, and second-order convergence of the manufactured
solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import box as X


def test_kron_assembly_is_the_seven_point_stencil():
    nx, ny, nz, h, kappa = 4, 3, 5, 0.25, -2.0
    A = X.box_operator(nx, ny, nz, h, kappa)
    p = np.random.default_rng(0).standard_normal((nz, ny, nx))
    q = np.pad(p, 1)  # zero one step beyond every face
    lap = (q[1:-1, 1:-1, 2:] + q[1:-1, 1:-1, :-2] + q[1:-1, 2:, 1:-1] + q[1:-1, :-2, 1:-1]
           + q[2:, 1:-1, 1:-1] + q[:-2, 1:-1, 1:-1] - 6 * p) / h ** 2
    assert np.allclose(A @ p.ravel(), (lap + kappa * p).ravel())
    assert abs(A - A.T).max() == 0.0


@pytest.mark.parametrize("abc", [(1, 1, 1), (4, 3, 5), (2, 1, 4)])
def test_eigenmodes(abc):
    nx, ny, nz, h, kappa = 4, 3, 5, 0.2, -1.0
    A = X.box_operator(nx, ny, nz, h, kappa)
    q = X.box_mode(*abc, nx, ny, nz)
    lam = X.box_eigenvalue(*abc, nx, ny, nz, h, kappa)
    assert np.allclose(A @ q, lam * q, atol=1e-10 * abs(lam))


def test_second_order_convergence():
    errs = []
    for n in (7, 15, 31):
        h, p, f = X.manufactured(n)
        z = spla.spsolve(X.box_operator(n, n, n, h).tocsc(), f)
        errs.append(np.abs(z - p).max())
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.8 < errs[1] / errs[2] < 4.2, errs


def test_direct_solve_equals_dst_banded_solve():
    """An independent route: scipy's DST-I along x and y, one banded solve per (kx, ky)
    along z, inverse DST -- equal to the sparse LU solve."""
    from scipy.fft import dstn, idstn
    from scipy.linalg import solve_banded
    nx, ny, nz, h, kappa = 5, 4, 6, 0.2, -1.0
    d = 1.0 / h ** 2
    v = np.random.default_rng(2).standard_normal((nz, ny, nx))
    V = dstn(v, type=1, axes=(1, 2))
    Z = np.empty_like(V)
    for ky in range(ny):
        for kx in range(nx):
            lam = (-4 * d * np.sin((kx + 1) * np.pi / (2 * (nx + 1))) ** 2
                   - 4 * d * np.sin((ky + 1) * np.pi / (2 * (ny + 1))) ** 2)
            ab = np.zeros((3, nz))
            ab[0, 1:] = d
            ab[1, :] = -2 * d + lam + kappa
            ab[2, :-1] = d
            Z[:, ky, kx] = solve_banded((1, 1), ab, V[:, ky, kx])
    z = idstn(Z, type=1, axes=(1, 2))
    want = X.solve_box(nx, ny, nz, h, kappa, v.ravel())[0]
    assert np.allclose(z.ravel(), want, rtol=1e-11, atol=1e-13)
