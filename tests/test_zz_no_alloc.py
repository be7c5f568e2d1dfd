"""fpg_fast_solve_noalloc: the fast solve for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).

Checked through the C ABI against the domain entry point fpg_block_solve on
the same inputs, call after call, at the FP64 tolerance of the other fast-solve
tests.  Kept in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _reference(B, n, kappa, v):
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=max(1, v.shape[0])))
    z = torch.zeros_like(v)
    d.block_solve(0, v, z, v.shape[0])
    torch.cuda.synchronize()
    out = z.cpu().numpy()
    d.close()
    return out


def test_noalloc_matches_block_solve_on_consecutive_calls(lib):
    from paper_2509_23180_gb300 import binding as B
    stream = torch.cuda.current_stream()
    # consecutive calls: same (n, kappa) twice (tables reused), then a new one
    for call, (n, kappa, nvec, seed) in enumerate([(64, -10.0, 5, 1), (64, -10.0, 3, 2), (256, 0.0, 4, 3),
                                                   (100, -1.0, 2, 4)]):
        v = torch.as_tensor(W.random_block_vectors(nvec, n * n, seed), device="cuda")
        z = torch.full_like(v, float("nan"))
        st = lib.fpg_fast_solve_noalloc(n, kappa, v.data_ptr(), z.data_ptr(), nvec, stream.cuda_stream)
        assert st == B.FPG_OK, (call, lib.fpg_last_cuda_error())
        torch.cuda.synchronize()
        got = z.cpu().numpy()
        want = _reference(B, n, kappa, v)
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-11, (call, err)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    from paper_2509_23180_gb300 import binding as B
    v = torch.zeros(4, device="cuda", dtype=torch.float64)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.fpg_fast_solve_noalloc(513, 0.0, v.data_ptr(), v.data_ptr(), 1, s) == B.FPG_EINVAL
    assert b"FPG_NOALLOC_MAX_N" in lib.fpg_last_cuda_error()
    assert lib.fpg_fast_solve_noalloc(512, 0.0, v.data_ptr(), v.data_ptr(), 9, s) == B.FPG_EINVAL
    assert b"FPG_NOALLOC_MAX_POINTS" in lib.fpg_last_cuda_error()
    assert lib.fpg_fast_solve_noalloc(64, 1.0, v.data_ptr(), v.data_ptr(), 1, s) == B.FPG_EINVAL
