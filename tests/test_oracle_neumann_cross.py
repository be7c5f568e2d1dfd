"""Pins of the Neumann-sided cross oracle (Sec. 3.1, Eq. "cross_equation"
boundary pattern; Eq. "submat_Neumann" closure) against facts that do not come
from its own assembly: face counts of the geometry, the two mirror symmetries
of the cross, negative definiteness, an arm block rebuilt from the Neumann
line operator and a Dirichlet-end sweep operator, the analytic solution's
boundary values and Laplacian by finite differences, and second-order
convergence."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import neumann as NM
from oracle import neumann_cross as X
from oracle.schur import BlockSystem, algorithm1


def test_cells_and_layout():
    n = 6
    pts = X.cells(n)
    assert len(pts) == 5 * n * n == len(set(pts))
    assert all(X.inside(I, J, n) for I, J in pts)
    # every inside cell of the bounding box [-n, 2n)^2 is listed
    box = {(I, J) for I in range(-n, 2 * n) for J in range(-n, 2 * n) if X.inside(I, J, n)}
    assert box == set(pts)
    xy = X.coordinates(n)
    assert xy.min() == pytest.approx(-1 + 0.5 / n) and xy.max() == pytest.approx(2 - 0.5 / n)


def test_face_counts_from_row_sums():
    """K 1 = kappa - 2 delta (#Dirichlet faces of the cell): with a Neumann face
    the row sum is unchanged, a Dirichlet face subtracts 2 delta.  The cross has
    4n Dirichlet faces (the far ends), one per end cell."""
    n, kappa = 7, -3.0
    K = X.assemble(n, kappa)
    d = float(n * n)
    rs = K @ np.ones(K.shape[0])
    nd = np.rint((kappa - rs) / (2 * d)).astype(int)
    assert np.allclose(rs, kappa - 2 * d * nd)
    assert nd.sum() == 4 * n and set(np.unique(nd)) == {0, 1}
    xy = X.coordinates(n)
    ends = (np.isclose(xy[:, 0], -1 + 0.5 / n) | np.isclose(xy[:, 0], 2 - 0.5 / n)
            | np.isclose(xy[:, 1], -1 + 0.5 / n) | np.isclose(xy[:, 1], 2 - 0.5 / n))
    assert np.array_equal(nd == 1, ends)
    # diagonal: -4 delta + kappa + delta (#Neumann faces) - delta (#Dirichlet faces);
    # Neumann faces: 8n arm-side faces in all
    nn = np.rint((K.diagonal() - (-4 * d + kappa)) / d).astype(int) + nd
    assert nn.sum() == 8 * n


def test_symmetric_negative_definite():
    for kappa in (0.0, -10.0):
        K = X.assemble(5, kappa).toarray()
        assert np.array_equal(K, K.T)
        assert np.linalg.eigvalsh(K).max() < 0


@pytest.mark.parametrize("mirror", ["swap_xy", "flip_x"])
def test_mirror_symmetry(mirror):
    """The cross and its boundary pattern are invariant under x <-> y and under
    x -> 1 - x; K commutes with the induced permutation of unknowns."""
    n = 6
    pts = X.cells(n)
    index = {p: k for k, p in enumerate(pts)}
    if mirror == "swap_xy":
        perm = [index[(J, I)] for I, J in pts]
    else:
        perm = [index[(n - 1 - I, J)] for I, J in pts]
    P = sp.csr_matrix((np.ones(len(pts)), (np.arange(len(pts)), perm)))
    K = X.assemble(n, -2.0)
    assert abs(P @ K @ P.T - K).max() == 0.0


def test_arm_block_from_line_operators():
    """The W block of K is  A^N_t (x) I + I (x) T_s + kappa I  with A^N_t the
    Neumann line operator along y and T_s = delta tridiag(1, -2, 1) along x whose
    first row (the far end x = -1) carries -3 delta."""
    n, kappa = 6, -4.0
    d = float(n * n)
    K = X.assemble(n, kappa)
    off = X.block_ranges(n)[1][5]
    KW = K[off:off + n * n, off:off + n * n].toarray()
    At = NM.neumann_line_operator(n, d)
    Ts = d * (np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1))
    Ts[0, 0] -= d
    want = np.kron(At, np.eye(n)) + np.kron(np.eye(n), Ts) + kappa * np.eye(n * n)
    assert np.allclose(KW, want, rtol=0, atol=1e-9 * d)


def test_analytic_solution_boundary_and_laplacian():
    t = np.array([-1.0, 0.0, 1.0, 2.0])
    assert np.allclose(X.psi(t) / np.pi, [0.0, 0.5, 1.5, 2.0])
    # derivatives against central differences
    s = np.linspace(-1, 2, 13)
    e = 1e-5
    assert np.allclose(X.dpsi(s), (X.psi(s + e) - X.psi(s - e)) / (2 * e), atol=1e-8)
    assert np.allclose(X.d2psi(s), (X.dpsi(s + e) - X.dpsi(s - e)) / (2 * e), atol=1e-7)
    # zero normal derivative on the arm sides, zero value at the far ends
    g = np.linspace(-1, 2, 7)
    for side in (0.0, 1.0):
        dy = (X.exact(g, side + e) - X.exact(g, side - e)) / (2 * e)
        assert np.abs(dy).max() < 1e-8
    for end in (-1.0, 2.0):
        assert np.abs(X.exact(end, np.linspace(0, 1, 5))).max() < 1e-12
    # the source is the Laplacian (+ kappa p) of the exact solution
    x, y, kappa, e = 0.3, -0.4, -2.5, 1e-4
    lap = (X.exact(x + e, y) + X.exact(x - e, y) + X.exact(x, y + e) + X.exact(x, y - e)
           - 4 * X.exact(x, y)) / e ** 2
    assert X.source(x, y, kappa) == pytest.approx(lap + kappa * X.exact(x, y), rel=1e-6)


def test_second_order_convergence():
    errs = []
    for n in (8, 16, 32):
        p, f = X.manufactured(n)
        z = spla.spsolve(X.assemble(n).tocsc(), f)
        errs.append(np.abs(z - p).max())
    assert 3.8 < errs[0] / errs[1] < 4.3 and 3.8 < errs[1] / errs[2] < 4.3, errs


def test_algorithm1_on_the_neumann_cross():
    """Alg. "fft_dd_solver" on the block pieces of this K reaches K^{-1} f."""
    n = 8
    K = X.assemble(n, -10.0)
    _, f = X.manufactured(n, -10.0)
    bs = BlockSystem(K, "cross", n, blocks=X.block_ranges(n))
    p, info = algorithm1(bs, f, m=20, rtol=1e-12)
    want = spla.spsolve(K.tocsc(), f)
    assert np.linalg.norm(p - want) / np.linalg.norm(want) < 1e-10


def test_workload_generator_agrees_with_oracle():
    """The input generator's restatement of the validation solution and source
    (monomial form) equals the oracle's (Newton form) at every cell centre."""
    import workloads as W
    for n, kappa in ((6, 0.0), (16, -3.0)):
        p, f = X.manufactured(n, kappa)
        assert np.allclose(W.ncross_validation_rhs(n, kappa), f, rtol=1e-13, atol=1e-12)
        assert np.allclose(W.ncross_validation_solution(n), p, rtol=1e-13, atol=1e-14)


def test_arms_couple_to_the_centre_only():
    """Each n x n arm touches the centre along one face of n cells and no other arm
    (the reentrant corners carry no unknown on the cell-centred grid)."""
    n = 6
    A = X.assemble(n, 0.0).tocsr()
    sl = {b[0]: slice(b[5], b[5] + b[6]) for b in X.block_ranges(n)}
    for a in ("W", "E", "S", "N"):
        for b in ("W", "E", "S", "N"):
            if a != b:
                assert A[sl[a], sl[b]].nnz == 0
        assert A[sl[a], sl["C"]].nnz == n
