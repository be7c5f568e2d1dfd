"""Pins for the block pieces, the Schur complement and Algorithm 1 (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from oracle import schur as S
from oracle import transforms as T


@pytest.fixture(scope="module")
def cross6():
    K = O.assemble("cross", 6, -10.0)
    return S.BlockSystem(K, "cross", 6)


def test_schur_is_inverse_of_global_inverse_block(cross6):
    """Block elimination: the Schur complement of the arms is the inverse of the
    centre block of K^{-1} (a textbook identity, independent of the code path)."""
    bs = cross6
    Kinv = np.linalg.inv(bs.K.toarray())
    c = bs.sl["C"]
    assert np.allclose(np.linalg.inv(Kinv[c, c]), bs.schur_dense(), rtol=1e-9, atol=1e-6)


def test_schur_symmetric_negative_definite(cross6):
    """L_c = A_c - sum R A^{-1} R^T is symmetric negative definite (the paper's
    remark that L_2 is not symmetric does not hold for this operator)."""
    L = cross6.schur_dense()
    assert np.allclose(L, L.T, rtol=1e-12, atol=1e-9)
    assert np.linalg.eigvalsh(L).max() < 0


def test_block_solve_on_an_arm_eigenmode(cross6):
    """A_W^{-1} of a rectangle mode is the mode over its eigenvalue."""
    n = 6
    nx, ny = W.block_shape("W", n)
    h = 1.0 / (n + 1)
    v = T.rectangle_mode(2, 3, nx, ny)
    lam = T.rectangle_eigenvalue(2, 3, nx, ny, h, -10.0)
    assert np.allclose(cross6.block_solve("W", v), v / lam, rtol=1e-12, atol=1e-15)


def test_schur_acts_only_on_the_lines_next_to_arms(cross6):
    """S = sum R_ca A_a^{-1} R_ac is nonzero only on C's lines that touch an arm."""
    n = 6
    Sd = cross6.A["C"].toarray() - cross6.schur_dense()
    rows = np.nonzero(np.abs(Sd).sum(axis=1) > 0)[0]
    i, j = rows % n, rows // n
    assert np.all((i == 0) | (i == n - 1) | (j == 0) | (j == n - 1))


@pytest.mark.parametrize("domain", ["cross", "T", "L"])
@pytest.mark.parametrize("kappa", [0.0, -10.0])
def test_algorithm1_equals_direct_solve(domain, kappa):
    """The Schur elimination is exact (Eq. "Schur_subeq"): Algorithm 1 run to a
    tight tolerance reproduces K^{-1} b."""
    n = 12
    K = O.assemble(domain, n, kappa)
    bs = S.BlockSystem(K, domain, n)
    f = W.fourier_rhs(domain, n, 5)
    p, info = S.algorithm1(bs, f, m=30, rtol=1e-13)
    ref = D.solve(K, f)
    assert info["converged"]
    assert np.linalg.norm(p - ref) < 1e-11 * np.linalg.norm(ref)


def test_preconditioner_cuts_iterations_sevenfold():
    """Sec. 3.2: with P = A_2^{-1} the iteration count to a fixed tolerance is
    more than seven times smaller than with P = I or the Jacobi P = D_2."""
    n = 24
    K = O.assemble("cross", n, 0.0)
    bs = S.BlockSystem(K, "cross", n)
    f = W.fourier_rhs("cross", n, 0)
    its = {}
    for pc in ("A_c", "none", "jacobi"):
        _, info = S.algorithm1(bs, f, m=30, rtol=1e-10, precond=pc, max_iters=2000)
        its[pc] = info["iterations"]
    assert 7 * its["A_c"] < its["none"] and 7 * its["A_c"] < its["jacobi"], its
