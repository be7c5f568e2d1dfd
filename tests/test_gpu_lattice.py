"""GPU parity of the general concatenated geometry (FPG_GEOM_LATTICE) against the
oracle (oracle/lattice.py): several coupled squares in arrangements whose
coupled set is not one rectangle -- a 2 x 2 block (four coupled squares, four
links, one junction), an L-shaped and a T-shaped coupled set with independent
squares, a ring of eight squares, the full 3 x 3 block, a domino and the cross.

Operator pieces element-wise (the coupled set's Schur matvec, the block-diagonal
preconditioner, K p), and whole solves against the oracle's direct solve
K^{-1} f: at rtol 1e-12 for small n, and at the workloads' rtol 1e-10 on 256^2
squares, with the residual re-checked with the oracle's K.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import direct as D
from oracle import lattice as LT
from tests.parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MASKS = dict(W.LATTICE_EXAMPLES)
MASKS["ring8"] = sum(1 << (i + 8 * j) for i in range(3) for j in range(3) if (i, j) != (1, 1))
MASKS["plus3x3"] = sum(1 << (i + 8 * j) for i in range(3) for j in range(3))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def domain(B, name, n, kappa, **kw):
    return B.Domain(B.make_desc("lattice", n, kappa, lattice=MASKS[name], **kw))


@pytest.mark.parametrize("name,n,kappa", [("square2x2", 9, 0.0), ("L5", 12, -10.0), ("T6", 7, -3.0),
                                          ("ring8", 6, 0.0), ("plus3x3", 5, -10.0), ("domino", 10, 0.0)])
def test_operator_pieces_vs_oracle(lib, name, n, kappa):
    """a2 (L_c z), a1 (the block-diagonal preconditioner) and a7 (K p)."""
    from paper_2509_23180_gb300 import binding as B
    mask = MASKS[name]
    K = LT.assemble(mask, n, kappa)
    bs, parts = LT.block_system(mask, n, K)
    nc = LT.coupled_size(mask, n)
    d = domain(B, name, n, kappa, nrhs=3)
    z = W.random_block_vectors(3, nc, seed=n)
    w = torch.zeros((3, nc), dtype=torch.float64, device="cuda")
    d.apply_schur(dev(z), 64, w, 3)
    assert rel(host(w), np.stack([bs.schur_apply(x) for x in z])) < 1e-11
    Ac = bs.A["C"].tocsc()
    want = np.zeros_like(z)
    for ix in parts:
        lu = spla.splu(Ac[ix][:, ix].tocsc())
        want[:, ix] = np.stack([lu.solve(x[ix]) for x in z])
    zz = torch.zeros((3, nc), dtype=torch.float64, device="cuda")
    d.apply_precond(dev(z), zz, 3)
    assert rel(host(zz), want) < 1e-11
    p = W.random_block_vectors(2, K.shape[0], seed=n + 1)
    y = torch.zeros((2, K.shape[0]), dtype=torch.float64, device="cuda")
    d.apply_global(dev(p), y, 2)
    assert rel(host(y), np.stack([K @ x for x in p])) < 1e-13
    d.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name,n,kappa", [("square2x2", 16, 0.0), ("L5", 20, -10.0), ("T6", 12, 0.0),
                                          ("ring8", 10, -10.0), ("plus3x3", 9, 0.0), ("domino", 24, -10.0),
                                          ("cross", 16, 0.0)])
def test_solve_vs_direct(lib, prec, name, n, kappa):
    from paper_2509_23180_gb300 import binding as B
    mask = MASKS[name]
    K = LT.assemble(mask, n, kappa)
    f = np.stack([W.lattice_fourier_rhs(mask, n, s) for s in (1, 2, 3)])
    ref = D.Factor(K).solve(f)
    d = domain(B, name, n, kappa, nrhs=3, restart=30, rtol=1e-12, precond_precision=prec)
    d.set_rhs(dev(f))
    p = torch.zeros((3, K.shape[0]), dtype=torch.float64, device="cuda")
    st, info = d.solve(p)
    assert st == B.FPG_OK, info
    P = host(p)
    for r in range(3):
        assert info[r]["residual"] <= 1e-12
        assert np.linalg.norm(f[r] - K @ P[r]) <= 1.01e-12 * np.linalg.norm(f[r])
        assert rel(P[r], ref[r]) < 1e-9, (name, r, rel(P[r], ref[r]))
    d.close()


def test_cross_arrangement_gives_the_cross_solution(lib):
    """The cross given as a lattice is the cross domain: same unknowns (renumbered),
    same solution."""
    from paper_2509_23180_gb300 import binding as B
    n, kappa = 20, -10.0
    m = n + 1
    mask = MASKS["cross"]
    lat = [(I - m, J - m) for I, J in LT.block_order_points(mask, n)]
    from oracle import geometry as G
    cro = G.block_order_points("cross", n)
    perm = np.array([cro.index(q) for q in lat])
    f_cross = W.rhs_batch("cross", n, [4], kind="fourier")
    dc = B.Domain(B.make_desc("cross", n, kappa, nrhs=1, rtol=1e-12))
    dc.set_rhs(dev(f_cross))
    pc = torch.zeros_like(dev(f_cross))
    assert dc.solve(pc)[0] == B.FPG_OK
    dl = domain(B, "cross", n, kappa, nrhs=1, rtol=1e-12)
    fl = f_cross[:, perm]
    dl.set_rhs(dev(fl))
    pl = torch.zeros_like(dev(fl))
    st, info = dl.solve(pl)
    assert st == B.FPG_OK
    assert rel(host(pl)[0], host(pc)[0][perm]) < 1e-10
    dc.close()
    dl.close()


@pytest.mark.parametrize("name,kappa", [("square2x2", 0.0), ("L5", -10.0)])
def test_bench_size_256_vs_oracle(lib, name, kappa):
    """256^2 per square, 4 RHS, FGMRES(30) at rtol 1e-10, element-wise against
    SuperLU, residual re-checked with the oracle's K."""
    from paper_2509_23180_gb300 import binding as B
    n = 256
    mask = MASKS[name]
    K = LT.assemble_grid(mask, n, kappa)
    f = np.stack([W.lattice_fourier_rhs(mask, n, s) for s in range(4)])
    ref = D.Factor(K).solve(f)
    d = domain(B, name, n, kappa, nrhs=4, restart=30, rtol=1e-10)
    d.set_rhs(dev(f))
    p = torch.zeros_like(dev(f))
    st, info = d.solve(p)
    assert st == B.FPG_OK, info
    P = host(p)
    for r in range(4):
        assert np.linalg.norm(f[r] - K @ P[r]) <= 1.01e-10 * np.linalg.norm(f[r])
        assert rel(P[r], ref[r]) < 1e-9
    d.close()


def test_identity_preconditioner_and_refusals(lib):
    from paper_2509_23180_gb300 import binding as B
    n = 8
    mask = MASKS["square2x2"]
    K = LT.assemble(mask, n, 0.0)
    f = W.lattice_fourier_rhs(mask, n, 5)[None, :]
    its = {}
    for kind in (0, 1):
        d = domain(B, "square2x2", n, 0.0, nrhs=1, rtol=1e-11, max_iters=5000)
        d.set_option(B.OPT_PRECOND, kind)
        d.set_rhs(dev(f))
        p = torch.zeros_like(dev(f))
        st, info = d.solve(p)
        assert st == B.FPG_OK
        assert rel(host(p)[0], D.solve(K, f[0])) < 1e-8
        its[kind] = info[0]["iterations"]
        if kind == 0:
            v = torch.zeros((1, n * n), dtype=torch.float64, device="cuda")
            assert lib.fpg_block_solve(d.handle, 0, v.data_ptr(), v.data_ptr(), 1) == B.FPG_EUNSUPPORTED
            assert lib.fpg_set_option(d.handle, B.OPT_PRECOND, 2) == B.FPG_EUNSUPPORTED
        d.close()
    assert its[0] < its[1]
    import ctypes
    out = ctypes.c_size_t()
    bad = B.make_desc("lattice", n, 0.0, lattice=(1 << 0) | (1 << 2))  # not edge-connected
    assert lib.fpg_workspace_bytes(ctypes.byref(bad), ctypes.byref(out)) == B.FPG_EINVAL
    # two spines joined at the top, three arms left and right of each: 12 independent
    # squares with a west or east neighbour, more than one batch of the arm kernels holds
    sq = {(c, j) for c in (1, 5) for j in range(8)} | {(2, 7), (3, 7), (4, 7)}
    sq |= {(c + dc, j) for c in (1, 5) for dc in (-1, 1) for j in (0, 2, 4)}
    many = sum(1 << (i + 8 * j) for i, j in sq)
    _, indep = LT.classify(many)
    assert sum(1 for d in indep.values() if d[1] == 0) == 12
    wide = B.make_desc("lattice", n, 0.0, lattice=many)
    assert lib.fpg_workspace_bytes(ctypes.byref(wide), ctypes.byref(out)) == B.FPG_EUNSUPPORTED
