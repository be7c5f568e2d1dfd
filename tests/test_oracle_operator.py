"""Pins for the oracle's operator K and direct solve (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import direct as D
from oracle import geometry as G
from oracle import operator as O
from oracle import transforms as T


@pytest.mark.parametrize("domain", ["cross", "T", "L"])
@pytest.mark.parametrize("kappa", [0.0, -10.0])
def test_K_symmetric_negative_definite(domain, kappa):
    """R_ij = R_ji^T (Sec. 2.3) makes K symmetric; with kappa <= 0 the 5-point
    operator is negative definite (so every A_i is invertible)."""
    K = O.assemble(domain, 6, kappa)
    assert abs(K - K.T).max() == 0.0
    ev = np.linalg.eigvalsh(K.toarray())
    assert ev.max() < 0.0


@pytest.mark.parametrize("nx,ny", [(5, 5), (7, 4), (4, 9)])
def test_centre_block_is_the_rectangle_operator(nx, ny):
    """The C block read off K equals the Kronecker form of Eq. "mat_Poisson"."""
    n = 8
    K = O.assemble("cross", n, -3.0)
    A = O.rectangle(n, n, 1.0 / (n + 1), -3.0)
    assert abs(K[: n * n, : n * n] - A).max() < 1e-9
    # and the rectangle operator of any shape has the textbook eigenpairs
    h = 0.1
    R = O.rectangle(nx, ny, h, -2.5)
    for k, l in [(1, 1), (nx, 1), (2, ny), (nx, ny)]:
        v = T.rectangle_mode(k, l, nx, ny)
        lam = T.rectangle_eigenvalue(k, l, nx, ny, h, -2.5)
        assert np.allclose(R @ v, lam * v, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("domain", ["cross", "T", "L"])
@pytest.mark.parametrize("n", [1, 2, 7, 24])
def test_grid_assembly_equals_pointwise_assembly(domain, n):
    """The grid-indexed K (used at n = 512 and 1024) is the point-by-point K:
    the same pattern and the same values, entry for entry."""
    A = O.assemble(domain, n, -10.0)
    B = O.assemble_grid(domain, n, -10.0)
    assert A.shape == B.shape
    A.sort_indices()
    B = B.tocsr()
    B.sort_indices()
    assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
    assert np.array_equal(A.data, B.data)


def test_five_point_stencil_is_exact_on_quadratics():
    """Away from the edge, (K q)_I = lap q + kappa q for any quadratic q
    (the central second difference is exact on quadratics)."""
    n = 10
    m = n + 1
    K = O.assemble("cross", n, -1.5)
    pts = G.block_order_points("cross", n)
    inside = set(pts)
    q = lambda x, y: 0.3 + 1.1 * x - 0.7 * y + 2.0 * x * x - 0.5 * x * y + 1.5 * y * y
    lap = 2.0 * 2.0 + 2.0 * 1.5
    vals = np.array([q(I / m, J / m) for I, J in pts])
    Kq = K @ vals
    for k, (I, J) in enumerate(pts):
        if all(nb in inside for nb in ((I + 1, J), (I - 1, J), (I, J + 1), (I, J - 1))):
            assert abs(Kq[k] - (lap - 1.5 * vals[k])) < 1e-8


def test_second_order_convergence_manufactured():
    """The discrete solution converges at O(h^2) to the manufactured p (the
    paper's accuracy claim, Sec. 3.1): the max error falls ~4x per halving of h."""
    errs = []
    for n in (15, 31, 63):
        K = O.assemble("cross", n, 0.0)
        p = D.solve(K, W.manufactured_rhs("cross", n, 0.0))
        errs.append(np.abs(p - W.manufactured_solution("cross", n)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_direct_dense_and_sparse_agree():
    n = 20
    K = O.assemble("cross", n, -10.0)
    b = W.fourier_rhs("cross", n, 1)
    x_sparse = D.Factor(K).solve(b)
    x_dense = np.linalg.solve(K.toarray(), b)
    assert np.abs(x_sparse - x_dense).max() < 1e-12 * np.abs(x_dense).max()
    assert O.global_residual(K, b, x_sparse) < 1e-14


def test_brute_force_tiny_inverse():
    """On a tiny cross the solve equals the explicit inverse applied to b."""
    n = 3
    K = O.assemble("cross", n, -10.0).toarray()
    b = W.fourier_rhs("cross", n, 2)
    x = D.solve(sp.csr_matrix(K), b)
    assert np.allclose(np.linalg.inv(K) @ b, x, rtol=1e-12, atol=1e-14)


def test_direct_batch_of_rhs_dense_and_sparse():
    """(nrhs, N) right-hand sides give the same rows as one-by-one solves."""
    for n in (4, 24):
        K = O.assemble("T", n, -1.0)
        b = np.stack([W.fourier_rhs("T", n, s) for s in (0, 1, 2)])
        F = D.Factor(K)
        X = F.solve(b)
        for r in range(3):
            assert np.allclose(X[r], F.solve(b[r]), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("case", ["cross64", "T40", "L30", "chain2_12", "ncross24", "periodic", "box"])
def test_library_direct_solve_equals_conjugate_gradient(case):
    """The library direct solves the oracle uses (dense LU, SuperLU) against a
    second route written from the textbook definition: CG on -K to a relative
    residual of 1e-12 (the rounding floor of the recurrence at n = 64 is ~5e-13)."""
    from oracle import box as Xb
    from oracle import neumann_cross as NC
    from oracle import periodic as P
    from oracle import strip as S
    rng = np.random.default_rng(11)
    if case == "cross64":
        K, b = O.assemble("cross", 64, 0.0), W.fourier_rhs("cross", 64, 1)
    elif case == "T40":
        K, b = O.assemble("T", 40, -10.0), W.fourier_rhs("T", 40, 2)
    elif case == "L30":
        K, b = O.assemble("L", 30, -3.0), W.fourier_rhs("L", 30, 3)
    elif case == "chain2_12":
        K, b = S.assemble(2, 12, -10.0), W.strip_fourier_rhs(2, 12, 4)
    elif case == "ncross24":
        K, b = NC.assemble(24, 0.0), W.ncross_fourier_rhs(24, 5)
    elif case == "periodic":
        K = P.rectangle_periodic_t(24, 17, 1 / 24, -1.0)
        b = rng.standard_normal(K.shape[0])
    else:
        K = Xb.box_operator(9, 8, 7, 0.1, -2.0)
        b = rng.standard_normal(K.shape[0])
    x_cg, steps = D.conjugate_gradient(K, b, rtol=1e-12)
    x = D.solve(K, b)
    assert np.linalg.norm(b - K @ x_cg) <= 1.5e-12 * np.linalg.norm(b), steps
    assert np.abs(x - x_cg).max() <= 1e-10 * np.abs(x).max()
