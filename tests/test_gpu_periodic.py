"""GPU parity of the periodic-rectangle fast solve (Sec. 2.2, Eq.
"submat_Periodic") against the periodic oracle: closed-form Hartley-type
modes, sparse direct solves on random inputs (odd and even n_t, ragged line
tiles), second-order convergence and the error codes."""
import ctypes

import numpy as np
import pytest

from oracle import periodic as P
from tests.parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




@pytest.mark.parametrize("nt,ns", [(2, 3), (8, 7), (15, 9), (64, 63), (256, 256), (1024, 100)])
def test_periodic_modes(lib, nt, ns):
    """A_P^{-1} of a mixture of cas(2 pi k j/nt) sin(l pi i/(ns+1)) modes (k = 0,
    the Nyquist mode and k, n-k pairs included) is the mixture over the closed-form
    eigenvalues."""
    from paper_2509_23180_gb300 import binding as B
    h, kappa = 1.0 / nt, -10.0
    rng = np.random.default_rng(nt + ns)
    kl = [(0, 1), (nt - 1, ns), (nt // 2, 1), (1, ns // 2 + 1), (min(3, nt - 1), 2)]
    v = np.zeros((2, nt * ns))
    want = np.zeros((2, nt * ns))
    for k, l in kl:
        q = P.rectangle_periodic_mode(k, l, nt, ns)
        lam = P.rectangle_periodic_eigenvalue(k, l, nt, ns, h, kappa)
        c = rng.standard_normal(2)
        v += c[:, None] * q
        want += (c / lam)[:, None] * q
    z = torch.zeros((2, nt * ns), dtype=torch.float64, device="cuda")
    B.periodic_solve(dev(v), z, nt, ns, h, kappa)
    assert rel(host(z), want) < 1e-11


@pytest.mark.parametrize("nt,ns,kappa", [(6, 5, 0.0), (9, 17, -10.0), (30, 17, -3.0), (14, 40, 0.0),
                                         (125, 33, -10.0), (256, 100, -1.0)])
def test_periodic_random_vs_oracle(lib, nt, ns, kappa):
    from paper_2509_23180_gb300 import binding as B
    h = 1.0 / nt
    v = np.random.default_rng(11).standard_normal((3, nt * ns))
    z = torch.zeros((3, nt * ns), dtype=torch.float64, device="cuda")
    B.periodic_solve(dev(v), z, nt, ns, h, kappa)
    assert rel(host(z), P.solve_periodic_rectangle(nt, ns, h, kappa, v)) < 1e-11


def test_periodic_second_order(lib):
    from paper_2509_23180_gb300 import binding as B
    errs = []
    for nt in (64, 128, 256):
        h, ns, p, f = P.manufactured(nt)
        z = torch.zeros((1, nt * ns), dtype=torch.float64, device="cuda")
        B.periodic_solve(dev(f[None, :]), z, nt, ns, h, 0.0)
        errs.append(np.max(np.abs(host(z)[0] - p)))
    assert 3.9 < errs[0] / errs[1] < 4.1 and 3.9 < errs[1] / errs[2] < 4.1, errs


def test_periodic_errors(lib):
    from paper_2509_23180_gb300 import binding as B
    nb = ctypes.c_size_t()
    assert lib.fpg_periodic_workspace_bytes(1, 4, 1, ctypes.byref(nb)) == B.FPG_EINVAL
    # 17 has a prime factor above 13: no FFT plan
    assert lib.fpg_periodic_workspace_bytes(17, 4, 1, ctypes.byref(nb)) == B.FPG_EUNSUPPORTED
    assert lib.fpg_periodic_workspace_bytes(18, 4, 1, ctypes.byref(nb)) == B.FPG_OK
    v = torch.zeros((1, 18 * 4), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(v)
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.fpg_periodic_solve(17, 4, 0.1, 0.0, v.data_ptr(), z.data_ptr(), 1, ws.data_ptr(), nb.value,
                                 st) == B.FPG_EUNSUPPORTED
    assert lib.fpg_periodic_solve(18, 4, 0.1, 0.0, v.data_ptr(), z.data_ptr(), 1, ws.data_ptr(), nb.value - 256,
                                 st) == B.FPG_ENOMEM
    assert lib.fpg_periodic_solve(18, 4, 0.1, 1.0, v.data_ptr(), z.data_ptr(), 1, ws.data_ptr(), nb.value,
                                 st) == B.FPG_EINVAL  # kappa > 0
    assert lib.fpg_periodic_solve(18, 4, 0.1, 0.0, v.data_ptr(), z.data_ptr(), 2, ws.data_ptr(), nb.value,
                                 st) == B.FPG_ENOMEM  # workspace sized for one rectangle
