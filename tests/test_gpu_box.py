"""GPU parity of the 3-D box fast solve (the 3-D extension after Sec. 2.1:
DST-I along x and y, Thomas along z) against the 7-point oracle: closed-form
eigenmodes, sparse direct solves on random inputs (non-cubic boxes, the dense,
Stockham, Rader and size-specialised DST engines), second-order convergence
and the plan's limits."""
import numpy as np
import pytest

from oracle import box as X
from tests.parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




@pytest.mark.parametrize("nx,ny,nz", [(2, 3, 1), (2, 2, 1), (8, 6, 5), (16, 16, 16), (64, 40, 9), (4096, 3, 2),
                                      (5, 4096, 2)])
def test_box_modes(lib, nx, ny, nz):
    from paper_2509_23180_gb300 import binding as B
    h, kappa = 1.0 / (nx + 1), -10.0
    modes = [(1, 1, 1), (nx, ny, nz), (nx // 2 + 1, 1, nz), (1, ny, (nz + 1) // 2)]
    rng = np.random.default_rng(nx * ny + nz)
    v = np.zeros((2, nx * ny * nz))
    want = np.zeros_like(v)
    for abc in modes:
        q = X.box_mode(*abc, nx, ny, nz)
        lam = X.box_eigenvalue(*abc, nx, ny, nz, h, kappa)
        c = rng.standard_normal(2)
        v += c[:, None] * q
        want += (c / lam)[:, None] * q
    plan = B.BoxPlan(nx, ny, nz, h, kappa, nvec=2)
    z = torch.zeros_like(dev(v))
    plan.solve(dev(v), z, 2)
    assert rel(host(z), want) < 1e-11
    plan.close()


@pytest.mark.parametrize("nx,ny,nz,kappa", [(7, 9, 4, 0.0), (12, 93, 3, -10.0), (100, 16, 6, -1.0),
                                            (64, 64, 20, 0.0), (256, 17, 3, -10.0)])
def test_box_random_vs_oracle(lib, nx, ny, nz, kappa):
    """nx + 1 = 8 (Stockham), 13 (radix 13), 101 (Rader), 65 and 257 (size-specialised
    where profitable); ny + 1 = 94 (dense DST), 17, 10, 65, 18."""
    from paper_2509_23180_gb300 import binding as B
    h = 1.0 / (max(nx, ny) + 1)
    v = np.random.default_rng(nx + ny + nz).standard_normal((3, nx * ny * nz))
    plan = B.BoxPlan(nx, ny, nz, h, kappa, nvec=3)
    z = torch.zeros_like(dev(v))
    plan.solve(dev(v), z, 3)
    assert rel(host(z), X.solve_box(nx, ny, nz, h, kappa, v)) < 1e-11
    plan.close()


def test_box_second_order(lib):
    from paper_2509_23180_gb300 import binding as B
    errs = []
    for n in (15, 31, 63):
        h, p, f = X.manufactured(n)
        plan = B.BoxPlan(n, n, n, h, 0.0, nvec=1)
        z = torch.zeros((1, n ** 3), dtype=torch.float64, device="cuda")
        plan.solve(dev(f[None, :]), z, 1)
        errs.append(np.abs(host(z)[0] - p).max())
        plan.close()
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.9 < errs[1] / errs[2] < 4.1, errs


def test_box_limits(lib):
    import ctypes
    from paper_2509_23180_gb300 import binding as B
    nb = ctypes.c_size_t()
    assert lib.fpg_box_plan_bytes(1, 4, 4, 1, ctypes.byref(nb)) == B.FPG_EINVAL
    assert lib.fpg_box_plan_bytes(4096, 4, 4, 17, ctypes.byref(nb)) == B.FPG_EINVAL  # nvec * nx > 65535
    plan = B.BoxPlan(4, 4, 4, 0.2, 0.0, nvec=1)
    v = torch.zeros((2, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(B.FpgError) as e:
        plan.solve(v, torch.zeros_like(v), 2)
    assert e.value.status == B.FPG_EINVAL
    plan.close()
