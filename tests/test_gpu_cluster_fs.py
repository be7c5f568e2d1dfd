"""The one-pass FP32 cluster fast solve (FPG_OPT_CLUSTER_FASTSOLVE) against the
oracle and against the three-kernel FP32 path.

a1 (Sec. 2.1): z = A_c^{-1} v on the centre block for n = 64 (a cluster of 2
CTAs) and n = 512 (16 CTAs), FP64 in and FP32 out; closed-form
eigenmodes; whole solves with the FP32 preconditioner against K^{-1} f.

FP32 bar of a fast solve: the FP32 line transforms round at u32 = 2^-24 per
operation, and the solution of a random right-hand side is dominated by the
lowest modes, which the transform's rounding reaches at about u32 log2(n)
relative; the tests take 2e-5 (n = 64) and 1e-4 (n = 512), and require the
cluster path to be no less accurate than the three-kernel FP32 path on the
same inputs (within a factor 2).
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from oracle import transforms as T
from tests.parity import assert_solution, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {64: 2e-5, 512: 1e-4}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def precond(B, n, kappa, v, cluster):
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=v.shape[0], precond_precision=32))
    d.set_option(B.OPT_CLUSTER_FASTSOLVE, cluster)
    assert d.fast_solve_path() == (7 if cluster else 1)
    z = torch.zeros((v.shape[0], n * n), dtype=torch.float32, device="cuda")  # the preconditioner's output type
    before = d.launch_count()
    d.apply_precond(dev(v), z, v.shape[0])
    torch.cuda.synchronize()
    launches = d.launch_count() - before
    d.close()
    return z.cpu().numpy().astype(np.float64), launches


@pytest.mark.parametrize("n,kappa", [(64, 0.0), (64, -10.0), (512, -10.0)])
def test_cluster_fast_solve_vs_oracle_and_three_kernel_path(lib, n, kappa):
    from paper_2509_23180_gb300 import binding as B
    nv = 5
    v = W.random_block_vectors(nv, n * n, seed=n + 3)
    A = O.rectangle(n, n, 1.0 / (n + 1), kappa)
    want = D.Factor(A).solve(v)
    zc, lc = precond(B, n, kappa, v, 1)
    z3, l3 = precond(B, n, kappa, v, 0)
    assert lc == 1 and l3 == 3, (lc, l3)  # one launch against three
    ec, e3 = rel(zc, want), rel(z3, want)
    assert ec < TOL[n] and ec <= 2.0 * e3 + 1e-7, (ec, e3)


@pytest.mark.parametrize("n", [64, 512])
def test_cluster_fast_solve_eigenmodes(lib, n):
    """A_c^{-1} of a rectangle mode is the mode over its closed-form eigenvalue
    (Eq. "Poisson_spectral_eigen"), including the lowest and highest modes."""
    from paper_2509_23180_gb300 import binding as B
    kappa = -10.0
    h = 1.0 / (n + 1)
    modes = [(1, 1), (n, n), (n // 2, 1), (1, n), (7, 3)]
    v = np.stack([T.rectangle_mode(k, l, n, n) for k, l in modes])
    want = np.stack([v[i] / T.rectangle_eigenvalue(k, l, n, n, h, kappa) for i, (k, l) in enumerate(modes)])
    z, _ = precond(B, n, kappa, v, 1)
    for i, mode in enumerate(modes):
        # a single mode in FP32: rounding leaks into the lowest modes, amplified by
        # cond(A_c) ~ 1 / sin^2(pi / 2(n+1)) relative to a high-mode input
        cond = 1.0 / np.sin(np.pi / (2 * (n + 1))) ** 2 * abs(
            T.rectangle_eigenvalue(*mode, n, n, h, kappa) / T.rectangle_eigenvalue(n, n, n, n, h, kappa))
        assert rel(z[i], want[i]) < max(TOL[n], 16 * 2.0 ** -24 * cond), (mode, rel(z[i], want[i]))


def test_cluster_fast_solve_batch_and_inactive_blocks_agree(lib):
    """Blocks are independent clusters: a block gives the same bits alone and in a batch."""
    from paper_2509_23180_gb300 import binding as B
    n = 512
    v = W.random_block_vectors(3, n * n, seed=11)
    zb, _ = precond(B, n, 0.0, v, 1)
    z1, _ = precond(B, n, 0.0, v[1:2], 1)
    assert np.array_equal(zb[1], z1[0])


@pytest.mark.parametrize("n,kappa,seeds", [(64, -10.0, [0, 1, 2]), (512, 0.0, [3, 4])])
def test_solves_with_the_cluster_preconditioner_match_the_oracle(lib, n, kappa, seeds):
    """FP64 FGMRES with the one-pass FP32 preconditioner reaches K^{-1} f element-wise."""
    from paper_2509_23180_gb300 import binding as B
    K = O.assemble_grid("cross", n, kappa)
    f = W.rhs_batch("cross", n, seeds, kind="fourier")
    ref = D.Factor(K).solve(f)
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=len(seeds), restart=40, rtol=1e-10, precond_precision=32))
    d.set_option(B.OPT_CLUSTER_FASTSOLVE, 1)
    assert d.fast_solve_path() == 7
    fd = dev(f)
    d.set_rhs(fd)
    p = torch.zeros_like(fd)
    st, info = d.solve(p)
    assert st == B.FPG_OK, info
    P = p.cpu().numpy()
    for r in range(len(seeds)):
        assert O.global_residual(K, f[r], P[r]) <= 1.01e-10
        assert_solution(P[r], ref[r], "cross", n, 1e-9)
    d.close()
