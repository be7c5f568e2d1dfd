"""GPU parity of the Neumann-rectangle fast solve (Sec. 2.2, Eq. "submat_Neumann")
against the Neumann oracle: closed-form eigenmodes, sparse direct solves on
random inputs, second-order convergence, and the error codes."""
import ctypes

import numpy as np
import pytest

from oracle import neumann as N
from tests.parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




@pytest.mark.parametrize("nt,ns", [(8, 7), (64, 63), (256, 256), (1024, 100)])
def test_neumann_modes(lib, nt, ns):
    """A_N^{-1} of a mixture of cos(k pi (j-1/2)/nt) sin(l pi i/(ns+1)) modes is
    the mixture over the closed-form eigenvalues (k = 0, the constant mode, included)."""
    from paper_2509_23180_gb300 import binding as B
    h, kappa = 1.0 / nt, -10.0
    rng = np.random.default_rng(nt)
    kl = [(0, 1), (nt - 1, ns), (nt // 2, 1), (1, ns // 2 + 1), (3, 2)]
    v = np.zeros((2, nt * ns))
    want = np.zeros((2, nt * ns))
    for k, l in kl:
        q = N.rectangle_neumann_mode(k, l, nt, ns)
        lam = N.rectangle_neumann_eigenvalue(k, l, nt, ns, h, kappa)
        c = rng.standard_normal(2)
        v += c[:, None] * q
        want += (c / lam)[:, None] * q
    z = torch.zeros((2, nt * ns), dtype=torch.float64, device="cuda")
    B.neumann_solve(dev(v), z, nt, ns, h, kappa)
    assert rel(host(z), want) < 1e-11


@pytest.mark.parametrize("nt,ns,kappa", [(6, 5, 0.0), (30, 17, -10.0), (14, 40, -3.0), (64, 63, 0.0),
                                         (256, 100, -10.0)])
def test_neumann_random_vs_oracle(lib, nt, ns, kappa):
    """Random inputs against the oracle's sparse direct solve; n_t = 30 and 14
    exercise radices 3, 5 and 7 of the FFT plan, n_s odd and even, ragged tiles."""
    from paper_2509_23180_gb300 import binding as B
    h = 1.0 / nt
    v = np.random.default_rng(7).standard_normal((3, nt * ns))
    z = torch.zeros((3, nt * ns), dtype=torch.float64, device="cuda")
    B.neumann_solve(dev(v), z, nt, ns, h, kappa)
    assert rel(host(z), N.solve_neumann_rectangle(nt, ns, h, kappa, v)) < 1e-11


def test_neumann_second_order(lib):
    """The GPU solution of the manufactured problem converges like h^2."""
    from paper_2509_23180_gb300 import binding as B
    errs = []
    for nt in (64, 128, 256):
        h, ns, p, f = N.manufactured(nt)
        z = torch.zeros((1, nt * ns), dtype=torch.float64, device="cuda")
        B.neumann_solve(dev(f[None, :]), z, nt, ns, h, 0.0)
        errs.append(np.max(np.abs(host(z)[0] - p)))
    assert 3.9 < errs[0] / errs[1] < 4.1 and 3.9 < errs[1] / errs[2] < 4.1, errs


def test_neumann_errors(lib):
    from paper_2509_23180_gb300 import binding as B
    nb = ctypes.c_size_t()
    assert lib.fpg_neumann_workspace_bytes(7, 4, 1, ctypes.byref(nb)) == B.FPG_EINVAL
    # 34 has a prime factor above 13: no FFT plan
    assert lib.fpg_neumann_workspace_bytes(34, 4, 1, ctypes.byref(nb)) == B.FPG_EUNSUPPORTED
    assert lib.fpg_neumann_workspace_bytes(36, 4, 1, ctypes.byref(nb)) == B.FPG_OK
    v = torch.zeros((1, 36 * 4), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(v)
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.fpg_neumann_solve(34, 4, 0.1, 0.0, v.data_ptr(), z.data_ptr(), 1, ws.data_ptr(), nb.value,
                                 st) == B.FPG_EUNSUPPORTED
    assert lib.fpg_neumann_solve(36, 4, 0.1, 0.0, v.data_ptr(), z.data_ptr(), 1, ws.data_ptr(), nb.value - 256,
                                 st) == B.FPG_ENOMEM
    assert lib.fpg_neumann_solve(36, 4, 0.1, 1.0, v.data_ptr(), z.data_ptr(), 1, ws.data_ptr(), nb.value,
                                 st) == B.FPG_EINVAL  # kappa > 0
    assert lib.fpg_neumann_solve(36, 4, 0.1, 0.0, v.data_ptr(), z.data_ptr(), 2, ws.data_ptr(), nb.value,
                                 st) == B.FPG_ENOMEM  # workspace sized for one rectangle
