"""GPU parity of the chain of crosses (several coupled blocks, Sec. 2.3-2.4)
against the chain oracle: the global operator, the block-diagonal
preconditioner of the coupled row, the Schur matvec with 2K + 2 arms, whole
solves against K^{-1} f (FP64 and FP32 preconditioner), the oracle's FGMRES
iteration count, batch and graph invariance, second-order convergence, and the
options a chain does not take."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from tests.parity import assert_solution, rel  # noqa: F401
from oracle import strip as X
from oracle.schur import BlockSystem, algorithm1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




def domain(B, K, n, kappa, **kw):
    return B.Domain(B.make_desc("chain", n, kappa, chain=K, **kw))


def parts(K, n):
    nxc = (2 * K - 1) * (n + 1) - 1
    return [np.array([j * nxc + c0 + x for j in range(n) for x in range(cnt)])
            for c0, cnt in X.centre_block_columns(K, n)]


@pytest.mark.parametrize("K,n", [(2, 5), (3, 16), (5, 8)])
def test_global_operator(lib, K, n):
    from paper_2509_23180_gb300 import binding as B
    A = X.assemble(K, n, -10.0)
    d = domain(B, K, n, -10.0, nrhs=2)
    p = W.random_block_vectors(2, A.shape[0], seed=K * n)
    y = torch.zeros_like(dev(p))
    d.apply_global(dev(p), y, 2)
    assert rel(host(y), np.stack([A @ pi for pi in p])) < 1e-13


@pytest.mark.parametrize("prec,tol", [(64, 1e-11), (32, 2e-5)])
@pytest.mark.parametrize("K,n", [(2, 8), (3, 64), (5, 16)])
def test_block_diagonal_preconditioner(lib, prec, tol, K, n):
    """a1 on the row with FPG_OPT_PRECOND = 3: the exact inverse of each square's
    own operator."""
    from paper_2509_23180_gb300 import binding as B
    A = X.assemble(K, n, -10.0)
    bs = BlockSystem(A, "chain", n, blocks=X.block_ranges(K, n))
    Ac = bs.A["C"].tocsc()
    nc = Ac.shape[0]
    d = domain(B, K, n, -10.0, nrhs=3, precond_precision=prec)
    d.set_option(B.OPT_PRECOND, 3)
    v = W.random_block_vectors(3, nc, seed=n + K)
    z = torch.zeros((3, nc), dtype=torch.float64 if prec == 64 else torch.float32, device="cuda")
    d.apply_precond(dev(v), z, 3)
    want = np.zeros_like(v)
    for ix in parts(K, n):
        lu = spla.splu(Ac[ix][:, ix].tocsc())
        want[:, ix] = np.stack([lu.solve(vi[ix]) for vi in v])
    assert rel(host(z).astype(np.float64), want) < tol


@pytest.mark.parametrize("K,n,kappa", [(2, 6, 0.0), (3, 31, -10.0), (5, 12, -3.0)])
def test_schur_matvec(lib, K, n, kappa):
    from paper_2509_23180_gb300 import binding as B
    A = X.assemble(K, n, kappa)
    bs = BlockSystem(A, "chain", n, blocks=X.block_ranges(K, n))
    nc = bs.A["C"].shape[0]
    d = domain(B, K, n, kappa, nrhs=2)
    zv = W.random_block_vectors(3, nc, seed=7 * n)
    w = torch.zeros((3, nc), dtype=torch.float64, device="cuda")
    d.apply_schur(dev(zv), 64, w, 3)
    assert rel(host(w), np.stack([bs.schur_apply(zi) for zi in zv])) < 1e-11


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("K,n,kappa", [(2, 8, 0.0), (3, 30, -10.0), (5, 17, 0.0), (2, 64, -10.0)])
def test_solve_vs_direct(lib, prec, K, n, kappa):
    from paper_2509_23180_gb300 import binding as B
    A = X.assemble(K, n, kappa)
    f = np.stack([W.strip_fourier_rhs(K, n, s) for s in (0, 1)] + [W.strip_manufactured_rhs(K, n, kappa)])
    lu = spla.splu(A.tocsc())
    d = domain(B, K, n, kappa, nrhs=3, rtol=1e-12, precond_precision=prec)
    d.set_rhs(dev(f))
    p = torch.zeros_like(dev(f))
    st, info = d.solve(p)
    assert st == B.FPG_OK, info
    P = host(p)
    for r in range(3):
        assert rel(P[r], lu.solve(f[r])) < 1e-9
        assert info[r]["residual"] <= 1e-12
        assert np.linalg.norm(f[r] - A @ P[r]) / np.linalg.norm(f[r]) <= 1.01e-12


def test_iterations_match_oracle_block_diagonal(lib):
    from paper_2509_23180_gb300 import binding as B
    K, n = 3, 16
    A = X.assemble(K, n, 0.0)
    f = W.strip_fourier_rhs(K, n, 4)
    bs = BlockSystem(A, "chain", n, blocks=X.block_ranges(K, n))
    _, oinfo = algorithm1(bs, f, m=30, rtol=1e-10, precond="block_diag", centre_parts=parts(K, n))
    d = domain(B, K, n, 0.0, nrhs=1, rtol=1e-10, restart=30)
    d.set_option(B.OPT_PRECOND, 3)
    d.set_rhs(dev(f[None, :]))
    p = torch.zeros_like(dev(f[None, :]))
    st, info = d.solve(p)
    assert st == B.FPG_OK
    assert abs(info[0]["iterations"] - oinfo["iterations"]) <= 1, (info[0], oinfo["iterations"])


def test_batch_and_graph_invariance(lib):
    from paper_2509_23180_gb300 import binding as B
    K, n = 3, 24
    f = np.stack([W.strip_fourier_rhs(K, n, s) for s in (5, 6, 7)])
    d3 = domain(B, K, n, -10.0, nrhs=3, rtol=1e-12)
    d3.set_rhs(dev(f))
    p3 = torch.zeros_like(dev(f))
    d3.solve(p3)
    d1 = domain(B, K, n, -10.0, nrhs=1, rtol=1e-12)
    d1.set_option(B.OPT_CUDA_GRAPHS, 0)
    for r in range(3):
        d1.set_rhs(dev(f[r:r + 1]))
        p1 = torch.zeros_like(dev(f[r:r + 1]))
        d1.solve(p1)
        assert rel(host(p1)[0], host(p3)[r]) < 1e-11


def test_second_order(lib):
    from paper_2509_23180_gb300 import binding as B
    errs = []
    for n in (31, 63, 127):
        f = W.strip_manufactured_rhs(2, n)[None, :]
        d = domain(B, 2, n, 0.0, nrhs=1, rtol=1e-12)
        d.set_rhs(dev(f))
        p = torch.zeros_like(dev(f))
        st, info = d.solve(p)
        assert st == B.FPG_OK
        errs.append(np.abs(host(p)[0] - W.strip_manufactured_solution(2, n)).max())
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.9 < errs[1] / errs[2] < 4.1, errs


def test_options_a_chain_does_not_take(lib):
    from paper_2509_23180_gb300 import binding as B
    d = domain(B, 2, 8, 0.0, nrhs=1)
    v = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(B.FpgError) as e:
        d.block_solve(1, v, torch.zeros_like(v), 1)
    assert e.value.status == B.FPG_EUNSUPPORTED
    with pytest.raises(B.FpgError) as e:
        d.autotune()
    assert e.value.status == B.FPG_EUNSUPPORTED
    with pytest.raises(B.FpgError) as e:
        d.set_option(B.OPT_PRECOND, 2)
    assert e.value.status == B.FPG_EUNSUPPORTED
    d.set_option(B.OPT_PRECOND, 1)  # the identity works on any length


def test_bench_configuration_residual(lib):
    """The bench's chain (K = 3, 256^2 per square, FGMRES(30), rtol 1e-10) with its
    launch configuration: the oracle's K, assembled independently, confirms the
    residual of every right-hand side (855,040 unknowns each)."""
    from paper_2509_23180_gb300 import binding as B
    K, n = 3, 256
    A = X.assemble(K, n, -10.0)
    f = np.stack([W.strip_fourier_rhs(K, n, s) for s in range(3)])
    d = domain(B, K, n, -10.0, nrhs=3, rtol=1e-10, restart=30)
    d.set_rhs(dev(f))
    p = torch.zeros_like(dev(f))
    st, info = d.solve(p)
    assert st == B.FPG_OK
    P = host(p)
    for r in range(3):
        res = np.linalg.norm(f[r] - A @ P[r]) / np.linalg.norm(f[r])
        # the oracle's plain sparse product rounds ~1e-12 worse than the library's
        # difference-form stencil at this size, hence the margins
        assert res <= 1.1e-10 and abs(res - info[r]["residual"]) <= 1e-11


@pytest.mark.parametrize("prec,tol", [(64, 1e-11), (32, 2e-5)])
def test_row_preconditioner(lib, prec, tol):
    """The default chain preconditioner: the coupled row's own operator (couplings
    between its squares included) inverted by one fast solve of the whole row,
    against the oracle's sparse solve with A_C; then whole solves reach K^{-1} f
    with the oracle's FGMRES iteration count for that preconditioner (+-1)."""
    from paper_2509_23180_gb300 import binding as B
    K, n = 3, 16
    A = X.assemble(K, n, -10.0)
    bs = BlockSystem(A, "chain", n, blocks=X.block_ranges(K, n))
    nc = bs.A["C"].shape[0]
    d = domain(B, K, n, -10.0, nrhs=2, precond_precision=prec, rtol=1e-10)
    v = W.random_block_vectors(2, nc, seed=9)
    z = torch.zeros((2, nc), dtype=torch.float64 if prec == 64 else torch.float32, device="cuda")
    d.apply_precond(dev(v), z, 2)
    assert rel(host(z).astype(np.float64), np.stack([bs.block_solve("C", vi) for vi in v])) < tol
    f = np.stack([W.strip_fourier_rhs(K, n, s) for s in (1, 2)])
    d.set_rhs(dev(f))
    p = torch.zeros_like(dev(f))
    st, info = d.solve(p)
    assert st == B.FPG_OK
    lu = spla.splu(A.tocsc())
    for r in range(2):
        assert rel(host(p)[r], lu.solve(f[r])) < 1e-8
        if prec == 64:
            _, oinfo = algorithm1(bs, f[r], m=30, rtol=1e-10, precond="A_c")
            assert abs(info[r]["iterations"] - oinfo["iterations"]) <= 1, (info[r], oinfo["iterations"])
    cross = B.Domain(B.make_desc("cross", 8, 0.0))
    with pytest.raises(B.FpgError) as e:
        cross.set_option(B.OPT_PRECOND, 3)
    assert e.value.status == B.FPG_EUNSUPPORTED
