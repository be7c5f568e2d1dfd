"""The three forms of the FP32 forward line DST give the same bits (FPG_OPT_DST_BULK):
0, the default streaming kernel (persistent, two CTAs per SM, bulk-copied FP64 rows,
packing straight from the staging buffer, in-place passes); 1, the persistent kernel
with one CTA per SM; 2, one CTA per tile.  They run the same arithmetic in the same
order, so the preconditioner output z = A_c^{-1} v (Sec. 2.1) must agree bit for bit,
for the lengths the streaming form covers (p = 513, 1025) and for two it does not
(p = 65 and p = 257, Rader: forms 0 and 2 are the per-tile kernel there).  The oracle comparison of
the default path is in test_gpu_parity.py and test_gpu_large.py; here the forms are
also checked against the oracle's fast solve once, element-wise.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from tests.parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def precond(B, n, v, form, active_all=True):
    d = B.Domain(B.make_desc("cross", n, -10.0, nrhs=v.shape[0], precond_precision=32))
    d.set_option(B.OPT_DST_BULK, form)
    z = torch.zeros((v.shape[0], n * n), dtype=torch.float32, device="cuda")
    d.apply_precond(torch.as_tensor(v, device="cuda"), z, v.shape[0])
    torch.cuda.synchronize()
    d.close()
    return z.cpu().numpy()


@pytest.mark.parametrize("n,nv", [(64, 7), (256, 3), (512, 5), (1024, 2)])
def test_forward_dst_forms_are_bit_identical(lib, n, nv):
    from paper_2509_23180_gb300 import binding as B
    v = W.random_block_vectors(nv, n * n, seed=n + nv)
    z0 = precond(B, n, v, 0)
    for form in (1, 2):
        assert np.array_equal(z0, precond(B, n, v, form)), (n, form)
    if n <= 512:
        A = O.rectangle(n, n, 1.0 / (n + 1), -10.0)
        want = D.Factor(A).solve(v)
        assert rel(z0.astype(np.float64), want) < 1e-4


def test_invalid_form_is_refused(lib):
    from paper_2509_23180_gb300 import binding as B
    d = B.Domain(B.make_desc("cross", 16, 0.0, nrhs=1))
    assert lib.fpg_set_option(d.handle, B.OPT_DST_BULK, 3) == B.FPG_EINVAL
    assert lib.fpg_set_option(d.handle, B.OPT_DST_BULK, 2) == B.FPG_OK
    d.close()
