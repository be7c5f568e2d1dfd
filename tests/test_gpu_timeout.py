"""Bounded device waits: a wait that runs out gives FPG_ETIMEOUT, not a trap or a hang.

The persistent forward DST kernels (FPG_OPT_DST_BULK forms 0, the default streaming
kernel, and 1) wait on an mbarrier for each line tile they fetch.  With FPG_OPT_WAIT_LIMIT = 0 every such wait gives up at once:
the kernel records it in the domain's status word, lets its copy in flight land
and returns.  The solve must then report FPG_ETIMEOUT for every right-hand side,
and the same domain, stream and context must solve correctly afterwards with
the default limit.  Nothing here faults the GPU: the copies are real and in
bounds, only the waiting is cut short.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from tests.parity import assert_solution

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("form,n", [(1, 64), (0, 512)])
def test_wait_that_runs_out_reports_etimeout_and_context_stays_usable(lib, form, n):
    """Form 1 (one CTA per SM) at n = 64 and form 0 (the default streaming kernel,
    p = 513) at n = 512.  After the forced give-up the same domain solves again with
    the default limit: at n = 64 the answer is checked against the oracle; at n = 512
    it must equal, bit for bit, a fresh domain's solve with the per-tile kernel
    (form 2, no waits), the forms being bit-identical."""
    from paper_2509_23180_gb300 import binding as B
    kappa = -10.0
    f = W.rhs_batch("cross", n, [1, 2], kind="fourier")
    fd = torch.as_tensor(f, device="cuda")
    desc = dict(nrhs=2, restart=20, rtol=1e-10, max_iters=400, precond_precision=32)
    d = B.Domain(B.make_desc("cross", n, kappa, **desc))
    d.set_option(B.OPT_DST_BULK, form)
    assert d.fast_solve_path() == 1  # the size-specialised line DST, whose FP32 forward waits on its copies
    d.set_option(B.OPT_WAIT_LIMIT, 0)
    d.set_rhs(fd)
    p = torch.zeros_like(fd)
    st, info = d.solve(p, check=False)
    torch.cuda.synchronize()  # the device is still answering
    assert st == B.FPG_ETIMEOUT, (st, info)
    assert all(i["status"] == B.FPG_ETIMEOUT for i in info)
    # default limit again: the same domain solves correctly
    d.set_option(B.OPT_WAIT_LIMIT, 1 << 22)
    d.set_rhs(fd)
    p.zero_()
    st, info = d.solve(p, check=False)
    assert st == B.FPG_OK, info
    P = p.cpu().numpy()
    if n <= 64:
        ref = D.Factor(O.assemble("cross", n, kappa)).solve(f)
        for r in range(2):
            assert_solution(P[r], ref[r], "cross", n, 1e-9)
    else:
        d2 = B.Domain(B.make_desc("cross", n, kappa, **desc))
        d2.set_option(B.OPT_DST_BULK, 2)
        d2.set_rhs(fd)
        p2 = torch.zeros_like(fd)
        assert d2.solve(p2, check=False)[0] == B.FPG_OK
        assert np.array_equal(P, p2.cpu().numpy())
        d2.close()
    d.close()


def test_wait_limit_option_is_validated(lib):
    from paper_2509_23180_gb300 import binding as B
    d = B.Domain(B.make_desc("cross", 16, 0.0, nrhs=1))
    assert lib.fpg_set_option(d.handle, B.OPT_WAIT_LIMIT, -1) == B.FPG_EINVAL
    assert lib.fpg_set_option(d.handle, B.OPT_WAIT_LIMIT, 1000) == B.FPG_OK
    d.close()
