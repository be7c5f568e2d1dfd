"""Pins of the chain oracle (several coupled blocks, Sec. 2.3-2.4): its block
listing against the interior points found from the squares alone, K = 1
against the cross oracle, the mirror symmetry x -> (2K-1) - x, second-order
convergence of the manufactured solution, and Alg. 1 with the block-diagonal
preconditioner of the coupled set against K^{-1} f."""
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
