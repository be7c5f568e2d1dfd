"""Pins for the general concatenated geometry (oracle/lattice.py; CPU only).

  * the block listing is exactly the set of grid points strictly inside the
    union of squares (found independently, point by point), each once, and the
    seeded-input module's layout lists the same points in the same order;
  * coupled / independent squares, links and junctions of sample arrangements
    follow the rule after Alg. "fft_dd_solver" (one neighbour: independent);
  * K is symmetric negative definite; on the cross arrangement it is the
    oracle's cross K up to the numbering of the unknowns; the grid assembly
    equals the point-by-point one;
  * second-order convergence to the manufactured solution (Sec. 3.1);
  * Alg. 1 with the block-diagonal preconditioner reproduces the dense solve.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import lattice as LT
from oracle import operator as O
from oracle import geometry as G
from oracle.schur import algorithm1

MASKS = W.LATTICE_EXAMPLES


@pytest.mark.parametrize("name", sorted(MASKS))
@pytest.mark.parametrize("n", [1, 3, 6])
def test_listing_is_the_interior_point_set(name, n):
    mask = MASKS[name]
    pts = LT.block_order_points(mask, n)
    assert len(pts) == len(set(pts))
    assert set(pts) == LT.interior_points(mask, n)
    # the input generator's layout: same blocks, same order
    lay = [(b[2], b[3], b[4], b[5]) for b in W.lattice_blocks(mask, n)]
    assert lay == [(b[1], b[2], b[3], b[4]) for b in LT.block_ranges(mask, n)]
    assert W.lattice_total_unknowns(mask, n) == len(pts)


def test_coupled_independent_links_junctions():
    c, a = LT.classify(MASKS["square2x2"])
    assert c == [(0, 0), (1, 0), (0, 1), (1, 1)] and a == {}
    assert LT.links(MASKS["square2x2"]) == [("V", 0, 0), ("V", 0, 1), ("H", 0, 0), ("H", 1, 0)]
    assert LT.junctions(MASKS["square2x2"]) == [(1, 1)]
    c, a = LT.classify(MASKS["L5"])
    assert c == [(0, 0), (1, 0), (0, 1)] and a == {(2, 0): (-1, 0), (0, 2): (0, -1)}
    assert LT.links(MASKS["L5"]) == [("V", 0, 0), ("H", 0, 0)] and LT.junctions(MASKS["L5"]) == []
    c, a = LT.classify(MASKS["cross"])
    assert c == [(1, 1)] and len(a) == 4 and LT.links(MASKS["cross"]) == []
    c, a = LT.classify(MASKS["domino"])
    assert c == [(0, 0)] and a == {(1, 0): (-1, 0)}
    assert LT.connected(MASKS["T6"]) and not LT.connected((1 << 0) | (1 << 2))


@pytest.mark.parametrize("name", sorted(MASKS))
def test_K_symmetric_negative_definite_and_grid_assembly(name):
    mask = MASKS[name]
    K = LT.assemble(mask, 4, -3.0)
    assert abs(K - K.T).max() == 0.0
    assert np.linalg.eigvalsh(K.toarray()).max() < 0.0
    Kg = LT.assemble_grid(mask, 4, -3.0)
    assert (K != Kg).nnz == 0


def test_cross_arrangement_is_the_cross():
    """The cross as a lattice (centre (1,1), arms around it) lists the same points
    as the cross geometry (shifted by one square) and has the same K."""
    n = 5
    m = n + 1
    lat = [(I - m, J - m) for I, J in LT.block_order_points(MASKS["cross"], n)]
    cro = G.block_order_points("cross", n)
    assert set(lat) == set(cro)
    perm = [cro.index(p) for p in lat]
    Kc = O.assemble("cross", n, -10.0).toarray()
    Kl = LT.assemble(MASKS["cross"], n, -10.0).toarray()
    assert np.array_equal(Kl, Kc[np.ix_(perm, perm)])


@pytest.mark.parametrize("name", ["square2x2", "L5"])
def test_second_order_convergence(name):
    mask = MASKS[name]
    errs = []
    for n in (7, 15, 31):
        p = D.solve(LT.assemble_grid(mask, n, 0.0), W.lattice_manufactured_rhs(mask, n, 0.0))
        errs.append(np.abs(p - W.lattice_manufactured_solution(mask, n)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs


@pytest.mark.parametrize("name", ["square2x2", "L5", "T6", "domino"])
@pytest.mark.parametrize("kappa", [0.0, -10.0])
def test_algorithm1_block_diagonal_reproduces_the_direct_solve(name, kappa):
    mask = MASKS[name]
    n = 6
    K = LT.assemble(mask, n, kappa)
    f = W.lattice_fourier_rhs(mask, n, 3)
    bs, parts = LT.block_system(mask, n, K)
    p, info = algorithm1(bs, f, m=20, rtol=1e-13, precond="block_diag", centre_parts=parts, max_iters=2000)
    want = np.linalg.solve(K.toarray(), f)
    assert np.abs(p - want).max() <= 1e-10 * np.abs(want).max()
    assert info["iterations"] > 0
    # the Schur complement is the inverse of K^{-1}'s coupled block
    nc = LT.coupled_size(mask, n)
    Kinv = np.linalg.inv(K.toarray())
    Lc = np.stack([bs.schur_apply(e) for e in np.eye(nc)], axis=1)
    assert np.allclose(Lc @ Kinv[:nc, :nc], np.eye(nc), atol=1e-9)
