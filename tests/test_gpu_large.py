"""GPU parity at the sizes the throughput targets are quoted on, element by element
against the FP64 oracle's direct solve p = K^{-1} f.

  * the 512^2-per-block cross (1,312,768 unknowns) with the FP32 preconditioner,
    a batch of right-hand sides (the batching workload's shape);
  * the 1024^2-per-block cross (5,246,976 unknowns), kappa = 0, FP32 DST/Thomas
    inside FP64 FGMRES(40) and the plain FP64 path (the precision workload);
  * a mixed L / T / cross batch with the FP32 preconditioner through
    fpg_solve_many.

The oracle assembles K from its grid index map (`operator.assemble_grid`, pinned
equal to the point-by-point assembly) and factors it with SuperLU (about 7 s at
n = 512 and 50 s at n = 1024).  Every solve runs at the workloads' rtol 1e-10;
the bar is the target's 1e-9 relative error, checked on the whole vector (2-norm
and max-abs) and on every block and interface line separately, and the global
residual is re-computed on the CPU with the oracle's K.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O
from tests.parity import assert_solution

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

_FACTORS = {}


def oracle(geom, n, kappa):
    key = (geom, n, kappa)
    if key not in _FACTORS:
        _FACTORS.clear()  # one large factor at a time (about 6 GB at n = 1024)
        K = O.assemble_grid(geom, n, kappa)
        _FACTORS[key] = (K, D.Factor(K))
    return _FACTORS[key]


def solve_gpu(B, geom, n, kappa, f, prec, restart):
    d = B.Domain(B.make_desc(geom, n, kappa, nrhs=f.shape[0], restart=restart, rtol=1e-10, precond_precision=prec))
    fd = torch.as_tensor(f, device="cuda")
    d.set_rhs(fd)
    p = torch.zeros_like(fd)
    st, info = d.solve(p, check=False)
    torch.cuda.synchronize()
    d.close()
    return st, info, p.cpu().numpy()


def check(B, geom, n, kappa, f, P, st, info, what):
    K, F = oracle(geom, n, kappa)
    ref = F.solve(f)
    assert st == B.FPG_OK, (what, info)
    for r in range(f.shape[0]):
        assert info[r]["residual"] <= 1e-10, (what, r, info[r])
        res = O.global_residual(K, f[r], P[r])
        assert res <= 1.01e-10, (what, r, res)
        assert_solution(P[r], ref[r], geom, n, 1e-9, what=f"{what} rhs {r}")


def test_cross512_fp32_preconditioner_batch_vs_oracle(lib):
    from paper_2509_23180_gb300 import binding as B
    n, kappa = 512, -10.0
    f = W.rhs_batch("cross", n, [0, 1, 2, 3], kind="fourier")
    st, info, P = solve_gpu(B, "cross", n, kappa, f, 32, 40)
    check(B, "cross", n, kappa, f, P, st, info, "cross 512 fp32 preconditioner")


@pytest.mark.parametrize("prec", [32, 64])
def test_cross1024_precision_workload_vs_oracle(lib, prec):
    """The precision workload: FP32 fast solve inside FP64 FGMRES(40), and the
    plain FP64 method, both against the same oracle solution."""
    from paper_2509_23180_gb300 import binding as B
    n, kappa = 1024, 0.0
    f = W.rhs_batch("cross", n, [0, 1], kind="fourier")
    st, info, P = solve_gpu(B, "cross", n, kappa, f, prec, 40)
    check(B, "cross", n, kappa, f, P, st, info, f"cross 1024 precond fp{prec}")


def test_mixed_batch_fp32_preconditioner_vs_oracle(lib):
    """A mixed L / T / cross batch (different n and kappa, FP32 preconditioner),
    solved together by fpg_solve_many, each instance against its oracle."""
    from paper_2509_23180_gb300 import binding as B
    cases = [("L", 256, 0.0, [5, 6]), ("T", 128, -10.0, [7, 8, 9]), ("cross", 512, 0.0, [10, 11])]
    doms, fs, ps = [], [], []
    for geom, n, kappa, seeds in cases:
        s = torch.cuda.Stream()
        d = B.Domain(B.make_desc(geom, n, kappa, nrhs=len(seeds), restart=40, rtol=1e-10, precond_precision=32),
                     stream=s)
        f = W.rhs_batch(geom, n, seeds, kind="fourier")
        fd = torch.as_tensor(f, device="cuda")
        torch.cuda.synchronize()
        d.set_rhs(fd)
        doms.append(d)
        fs.append(f)
        ps.append(torch.zeros_like(fd))
    st, infos = B.solve_many(doms, ps)
    torch.cuda.synchronize()
    for (geom, n, kappa, _), f, p, info in zip(cases, fs, ps, infos):
        check(B, geom, n, kappa, f, p.cpu().numpy(), st, info, f"mixed {geom} {n}")
    for d in doms:
        d.close()
