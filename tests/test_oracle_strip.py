"""Pins of the chain oracle (several coupled blocks, Sec. 2.3-2.4): its block
listing against the interior points found from the squares alone, K = 1
against the cross oracle, the mirror symmetry x -> (2K-1) - x, second-order
convergence of the manufactured solution, the coupled row's own operator
against the Dirichlet rectangle and its DST-I inverse, and Alg. 1 with the row
and the block-diagonal preconditioner of the coupled set against K^{-1} f."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import operator as O
from oracle import strip as X
from oracle.schur import BlockSystem, algorithm1


@pytest.mark.parametrize("K,n", [(1, 4), (2, 5), (3, 3), (4, 2)])
def test_listing_is_the_interior(K, n):
    pts = X.block_order_points(K, n)
    assert len(pts) == len(set(pts)) == W.strip_total_unknowns(K, n)
    assert set(pts) == X.interior_points(K, n)


def test_K1_is_the_cross():
    n = 6
    assert abs(X.assemble(1, n, -3.0) - O.assemble("cross", n, -3.0)).max() == 0.0


@pytest.mark.parametrize("K", [2, 3])
def test_mirror_symmetry(K):
    n = 4
    m = n + 1
    pts = X.block_order_points(K, n)
    index = {p: k for k, p in enumerate(pts)}
    perm = [index[((2 * K - 1) * m - I, J)] for I, J in pts]
    P = sp.csr_matrix((np.ones(len(pts)), (np.arange(len(pts)), perm)))
    A = X.assemble(K, n, -1.0)
    assert abs(P @ A @ P.T - A).max() == 0.0


def test_second_order_convergence():
    errs = []
    for n in (7, 15, 31):
        f = W.strip_manufactured_rhs(2, n)
        z = spla.spsolve(X.assemble(2, n).tocsc(), f)
        errs.append(np.abs(z - W.strip_manufactured_solution(2, n)).max())
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.8 < errs[1] / errs[2] < 4.2, errs


@pytest.mark.parametrize("K", [2, 3])
def test_algorithm1_block_diagonal(K):
    n, kappa = 6, -10.0
    A = X.assemble(K, n, kappa)
    bs = BlockSystem(A, "strip", n, blocks=X.block_ranges(K, n))
    nxc = (2 * K - 1) * (n + 1) - 1
    parts = [np.array([j * nxc + c0 + x for j in range(n) for x in range(cnt)])
             for c0, cnt in X.centre_block_columns(K, n)]
    assert sorted(np.concatenate(parts)) == list(range(nxc * n))
    f = W.strip_fourier_rhs(K, n, 1)
    p, info = algorithm1(bs, f, m=30, rtol=1e-12, precond="block_diag", centre_parts=parts)
    want = spla.spsolve(A.tocsc(), f)
    assert np.linalg.norm(p - want) / np.linalg.norm(want) < 1e-10
    assert info["converged"]


def test_arms_are_independent_blocks():
    """Sec. 2.4's rule: every arm touches one block only (the coupled row), along
    exactly n of its unknowns (its interface line), and no two arms touch."""
    K, n = 3, 5
    A = X.assemble(K, n, 0.0).tocsr()
    blocks = X.block_ranges(K, n)
    sl = {b[0]: slice(b[5], b[5] + b[6]) for b in blocks}
    arms = [b[0] for b in blocks if b[0] != "C"]
    for a in arms:
        for b in arms:
            if a != b:
                assert A[sl[a], sl[b]].nnz == 0, (a, b)
        coupling = A[sl[a], sl["C"]]
        assert coupling.nnz == n                      # one neighbour per interface node
        assert len(set(coupling.nonzero()[0])) == n   # on n distinct arm unknowns


def test_row_block_is_the_dirichlet_rectangle_and_its_dst_inverse():
    """The coupled row's own operator A_C (read off K) is the 5-point Dirichlet
    rectangle of nx_c x n points built from 1-D operators, and its inverse is the
    double DST-I eigen-solve (scipy's DST, an independent route)."""
    from scipy.fft import dstn, idstn
    K, n, kappa = 2, 5, -7.0
    nxc = (2 * K - 1) * (n + 1) - 1
    d = float((n + 1) ** 2)
    T = lambda m: d * sp.diags([np.ones(m - 1), -2.0 * np.ones(m), np.ones(m - 1)], [-1, 0, 1])
    A_rect = sp.kron(sp.identity(n), T(nxc)) + sp.kron(T(n), sp.identity(nxc)) + kappa * sp.identity(nxc * n)
    bs = BlockSystem(X.assemble(K, n, kappa), "strip", n, blocks=X.block_ranges(K, n))
    assert abs(bs.A["C"] - A_rect).max() == 0.0
    v = np.random.default_rng(4).standard_normal(nxc * n)
    lam_x = -4.0 * d * np.sin(np.arange(1, nxc + 1) * np.pi / (2 * (nxc + 1))) ** 2
    lam_y = -4.0 * d * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
    V = dstn(v.reshape(n, nxc), type=1)
    z = idstn(V / (lam_y[:, None] + lam_x[None, :] + kappa), type=1).ravel()
    assert np.abs(bs.block_solve("C", v) - z).max() < 1e-12 * np.abs(z).max()


@pytest.mark.parametrize("K", [2, 3])
def test_algorithm1_row_preconditioner(K):
    """The default preconditioner of the coupled set (one solve of the whole
    row) reaches K^{-1} f, in fewer GMRES steps than the block diagonal of the
    squares, which leaves the couplings between squares to the Krylov loop."""
    n, kappa = 6, -10.0
    A = X.assemble(K, n, kappa)
    bs = BlockSystem(A, "strip", n, blocks=X.block_ranges(K, n))
    nxc = (2 * K - 1) * (n + 1) - 1
    parts = [np.array([j * nxc + c0 + x for j in range(n) for x in range(cnt)])
             for c0, cnt in X.centre_block_columns(K, n)]
    f = W.strip_fourier_rhs(K, n, 1)
    want = spla.spsolve(A.tocsc(), f)
    p, info = algorithm1(bs, f, m=30, rtol=1e-12)
    assert info["converged"] and np.linalg.norm(p - want) / np.linalg.norm(want) < 1e-10
    _, info_bd = algorithm1(bs, f, m=30, rtol=1e-12, precond="block_diag", centre_parts=parts)
    assert info["iterations"] < info_bd["iterations"]
