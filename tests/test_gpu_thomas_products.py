"""The FP64 Thomas sweeps with the tabulated carry products (FPG_OPT_THOMAS_PRODUCTS,
default) and with the products formed in the kernel give the same bits: the tables hold
the same products, multiplied on the host in the kernel's order (Sec. 2.1, the mode-k
tridiagonal solves of Eq. "trans_subeq").  Checked on the centre preconditioner (chunks
of 1, 2 and 8 rows), on the arms (chunks of 9 rows, sweeps of n + 1) through whole
solves, and against the oracle once."""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from tests.parity import rel, assert_solution

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,nv", [(16, 3), (40, 2), (256, 4)])
def test_precond_with_and_without_products_same_bits(lib, n, nv):
    from paper_2509_23180_gb300 import binding as B
    v = W.random_block_vectors(nv, n * n, seed=n)
    out = {}
    for use in (1, 0):
        d = B.Domain(B.make_desc("cross", n, -10.0, nrhs=nv))
        d.set_option(B.OPT_THOMAS_PRODUCTS, use)
        z = torch.zeros((nv, n * n), dtype=torch.float64, device="cuda")
        d.apply_precond(dev(v), z, nv)
        torch.cuda.synchronize()
        out[use] = z.cpu().numpy()
        d.close()
    assert np.array_equal(out[0], out[1])
    A = O.rectangle(n, n, 1.0 / (n + 1), -10.0)
    assert rel(out[1], D.Factor(A).solve(v)) < 1e-11


@pytest.mark.parametrize("geom,n", [("cross", 64), ("T", 256)])
def test_whole_solves_same_bits(lib, geom, n):
    from paper_2509_23180_gb300 import binding as B
    f = W.rhs_batch(geom, n, [3, 4], kind="fourier")
    fd = dev(f)
    P = {}
    for use in (1, 0):
        d = B.Domain(B.make_desc(geom, n, 0.0, nrhs=2, rtol=1e-10))
        d.set_option(B.OPT_THOMAS_PRODUCTS, use)
        d.set_rhs(fd)
        p = torch.zeros_like(fd)
        st, info = d.solve(p)
        assert st == B.FPG_OK, info
        P[use] = p.cpu().numpy()
        d.close()
    assert np.array_equal(P[0], P[1])
    if n <= 64:
        ref = D.Factor(O.assemble(geom, n, 0.0)).solve(f)
        for r in range(2):
            assert_solution(P[1][r], ref[r], geom, n, 1e-9)


def test_option_is_validated(lib):
    from paper_2509_23180_gb300 import binding as B
    d = B.Domain(B.make_desc("cross", 16, 0.0, nrhs=1))
    assert lib.fpg_set_option(d.handle, B.OPT_THOMAS_PRODUCTS, 2) == B.FPG_EINVAL
    assert lib.fpg_set_option(d.handle, B.OPT_THOMAS_PRODUCTS, 0) == B.FPG_OK
    d.close()
