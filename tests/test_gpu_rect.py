"""GPU parity of the rectangle fast-solve plans (Sec. 2.1-2.2: DST-I,
DCT-II and real-DFT lines) against the oracle's sparse direct solves, with
n_t != n_s, several solves per plan, ragged batches and the plan's limits."""
import numpy as np
import pytest

from oracle import neumann as NM
from tests.parity import rel
from oracle import operator as O
from oracle import periodic as PD

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




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
                                        ("periodic", 45, 70), ("periodic", 512, 64),
                                        # sweeps longer than the register Thomas kernel holds
                                        ("dirichlet", 64, 2000), ("neumann", 32, 1500), ("periodic", 24, 3001)])
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


@pytest.mark.parametrize("kind,nt,ns", [("neumann", 2048, 4096), ("periodic", 2048, 300), ("dirichlet", 4096, 64),
                                        ("neumann", 2, 1), ("periodic", 2, 1), ("dirichlet", 2, 1)])
def test_rect_plan_extreme_sizes(lib, kind, nt, ns):
    """The largest and smallest accepted shapes, checked on closed-form modes
    (the oracle's sparse solve of 8.4M unknowns would not finish in seconds)."""
    from paper_2509_23180_gb300 import binding as B
    h, kappa = 1.0 / nt, -3.0
    if kind == "neumann":
        mode, lam = NM.rectangle_neumann_mode, NM.rectangle_neumann_eigenvalue
        ks = [0, nt - 1, nt // 2]
    elif kind == "periodic":
        mode, lam = PD.rectangle_periodic_mode, PD.rectangle_periodic_eigenvalue
        ks = [0, nt - 1, nt // 2]
    else:
        from oracle import transforms as T
        mode = lambda k, l, a, b: T.rectangle_mode(k, l, a, b)
        lam = lambda k, l, a, b, hh, kk: T.rectangle_eigenvalue(k, l, a, b, hh, kk)
        ks = [1, nt, nt // 2]
    v = np.zeros(nt * ns)
    want = np.zeros(nt * ns)
    for i, k in enumerate(ks):
        l = [1, ns, (ns + 1) // 2][i]
        q = mode(k, l, nt, ns)
        v += (i + 1) * q
        want += (i + 1) / lam(k, l, nt, ns, h, kappa) * q
    plan = B.RectPlan(kind, nt, ns, h, kappa, nvec=1)
    z = torch.zeros((1, nt * ns), dtype=torch.float64, device="cuda")
    plan.solve(dev(v[None, :]), z, 1)
    assert rel(host(z)[0], want) < 1e-10
    plan.solve(dev(v[None, :]), z, 0)  # an empty batch launches nothing
    plan.close()
