"""fpg_fast_solve_noalloc: the fast solve for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).

Such callers run inside another framework's memory pool, or on a path whose
device memory was reserved up front, and cannot hand fpg_create_domain a
workspace.  The entry point is checked through the C ABI, call after call:
against the domain entry point fpg_block_solve on the same inputs, and against
the oracle's plain definition z = A^{-1} v (a sparse LU of the n x n Dirichlet
rectangle operator), at the FP64 fast-solve tolerance of the other tests.  The
calls cover every DST plan kind (Stockham, Rader, the dense fallback), the
largest batch the array holds, and a return to an earlier (n, kappa) after the
tables were replaced.  Kept in a file that pytest collects last.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from tests.parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _block_solve(B, n, kappa, v):
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=max(1, v.shape[0])))
    z = torch.zeros_like(v)
    d.block_solve(0, v, z, v.shape[0])
    torch.cuda.synchronize()
    out = z.cpu().numpy()
    d.close()
    return out


def _oracle(n, kappa, v):
    A = O.rectangle(n, n, 1.0 / (n + 1), kappa)
    return D.Factor(A).solve(v)


# (n, kappa, nvec, seed): p = n + 1 = 65 (Stockham), twice in a row (tables
# reused), 257 (Rader), 101 (Rader), 94 = 2 * 47 (dense fallback), 513 with
# nvec * n * n = FPG_NOALLOC_MAX_POINTS (the whole coefficient area and the
# largest table region), then back to the first (n, kappa)
CALLS = [(64, -10.0, 5, 1), (64, -10.0, 3, 2), (256, 0.0, 4, 3), (100, -1.0, 2, 4), (93, 0.0, 2, 5),
         (512, -10.0, 8, 6), (64, -10.0, 2, 7)]


def test_noalloc_matches_block_solve_and_oracle_on_consecutive_calls(lib):
    from paper_2509_23180_gb300 import binding as B
    stream = torch.cuda.current_stream()
    for call, (n, kappa, nvec, seed) in enumerate(CALLS):
        vh = W.random_block_vectors(nvec, n * n, seed)
        v = torch.as_tensor(vh, device="cuda")
        z = torch.full_like(v, float("nan"))
        st = lib.fpg_fast_solve_noalloc(n, kappa, v.data_ptr(), z.data_ptr(), nvec, stream.cuda_stream)
        assert st == B.FPG_OK, (call, lib.fpg_last_cuda_error())
        torch.cuda.synchronize()
        got = z.cpu().numpy()
        assert np.isfinite(got).all(), call
        want = _block_solve(B, n, kappa, v)
        assert rel(got, want) < 1e-11, (call, rel(got, want))
        err = rel(got, _oracle(n, kappa, vh))
        assert err < 1e-11, (call, err)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    from paper_2509_23180_gb300 import binding as B
    v = torch.zeros(4, device="cuda", dtype=torch.float64)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.fpg_fast_solve_noalloc(513, 0.0, v.data_ptr(), v.data_ptr(), 1, s) == B.FPG_EINVAL
    assert b"FPG_NOALLOC_MAX_N" in lib.fpg_last_cuda_error()
    assert lib.fpg_fast_solve_noalloc(512, 0.0, v.data_ptr(), v.data_ptr(), 9, s) == B.FPG_EINVAL
    assert b"FPG_NOALLOC_MAX_POINTS" in lib.fpg_last_cuda_error()
    # n = 2 leaves room for 2^19 vectors in the array; the batch is capped first
    assert lib.fpg_fast_solve_noalloc(2, 0.0, v.data_ptr(), v.data_ptr(), 4097, s) == B.FPG_EINVAL
    assert b"FPG_NOALLOC_MAX_NVEC" in lib.fpg_last_cuda_error()
    assert lib.fpg_fast_solve_noalloc(64, 1.0, v.data_ptr(), v.data_ptr(), 1, s) == B.FPG_EINVAL
