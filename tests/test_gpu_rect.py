"""GPU parity of the rectangle fast-solve plans (Sec. 2.1-2.2: DST-I,
DCT-II and real-DFT lines) against the oracle's sparse direct solves, with
n_t != n_s, several solves per plan, ragged batches and the plan's limits."""
import numpy as np
import pytest

from oracle import neumann as NM
from oracle import operator as O
from oracle import periodic as PD

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_solve(kind, nt, ns, h, kappa, v):
    import scipy.sparse.linalg as spla
    if kind == "dirichlet":
        A = O.rectangle(nt, ns, h, kappa)
    elif kind == "neumann":
        A = NM.rectangle_neumann_t(nt, ns, h, kappa)
    else:
        A = PD.rectangle_periodic_t(nt, ns, h, kappa)
    lu = spla.splu(A.tocsc())
    return np.stack([lu.solve(x) for x in v])


@pytest.mark.parametrize("kind,nt,ns", [("dirichlet", 64, 40), ("dirichlet", 93, 17), ("dirichlet", 256, 257),
                                        ("neumann", 64, 40), ("neumann", 90, 33), ("periodic", 64, 40),
                                        ("periodic", 45, 70), ("periodic", 512, 64)])
def test_rect_plan_vs_oracle(lib, kind, nt, ns):
    from paper_2509_23180_gb300 import binding as B
    h, kappa = 1.0 / nt, -5.0
    plan = B.RectPlan(kind, nt, ns, h, kappa, nvec=5)
    for seed, nv in ((1, 5), (2, 3)):  # the plan serves several solves, ragged batches
        v = np.random.default_rng(seed + nt).standard_normal((nv, nt * ns))
        z = torch.zeros((nv, nt * ns), dtype=torch.float64, device="cuda")
        plan.solve(dev(v), z, nv)
        assert rel(host(z), oracle_solve(kind, nt, ns, h, kappa, v)) < 1e-11, (kind, seed)
    plan.close()


def test_rect_plan_limits(lib):
    from paper_2509_23180_gb300 import binding as B
    plan = B.RectPlan("neumann", 16, 8, 0.1, 0.0, nvec=2)
    v = torch.zeros((3, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(B.FpgError) as e:
        plan.solve(v, torch.zeros_like(v), 3)  # more rectangles than the plan holds
    assert e.value.status == B.FPG_EINVAL
    plan.close()
