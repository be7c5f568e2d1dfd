"""The library's batch runtime (fpg_batch_*): requests of mixed descriptors
(all-Dirichlet L/T/cross, the Neumann-sided cross, a chain) solved by
continuous batching over resident domains, each result against K^{-1} f of
its oracle; coalescing of a key's pending requests, eviction when the pool is
short, refusal over budget, and the serving loop on top of it."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from tests.parity import assert_solution, rel  # noqa: F401
from oracle import neumann_cross as NX
from oracle import operator as O
from oracle import strip as SX

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




def run(batch, live, limit=200000):
    """Step until every ticket of `live` is done; returns {ticket: info}."""
    out = {}
    for _ in range(limit):
        finished = set(batch.step())
        for t, nr in list(live.items()):
            info = batch.poll(t, nr)
            assert (info is not None) == (t in finished)  # step reports exactly the tickets it finished
            if info is not None:
                out[t] = info
                del live[t]
        if not live:
            return out
    raise AssertionError("batch runtime did not finish")


def test_mixed_requests_match_direct_solves(lib):
    from paper_2509_23180_gb300 import binding as B
    cases = []  # (desc, f, K)
    for geom, n, kappa in (("cross", 24, 0.0), ("L", 17, -10.0), ("T", 20, -3.0), ("cross", 24, 0.0)):
        f = W.rhs_batch(geom, n, [len(cases), len(cases) + 1], kind="fourier")
        cases.append((B.make_desc(geom, n, kappa, nrhs=2, rtol=1e-12), f, O.assemble(geom, n, kappa)))
    n = 16
    f = np.stack([W.ncross_fourier_rhs(n, 3)])
    cases.append((B.make_desc("cross", n, -10.0, nrhs=1, rtol=1e-12, boundary="neumann_sides"), f,
                  NX.assemble(n, -10.0)))
    f = np.stack([W.strip_fourier_rhs(2, 12, s) for s in (1, 2, 3)])
    cases.append((B.make_desc("chain", 12, 0.0, nrhs=3, rtol=1e-12, chain=2), f, SX.assemble(2, 12, 0.0)))
    batch = B.Batch(4 << 30, slots=4, max_domains=16)
    live, bufs = {}, {}
    for desc, f, A in cases:
        fd = dev(f)
        p = torch.zeros_like(fd)
        t = batch.admit(desc, fd, p)
        live[t] = desc.nrhs
        bufs[t] = (fd, p, f, A)
    infos = run(batch, live)
    st = batch.stats()
    assert st["created"] == 5 and st["open_tickets"] == 0  # the two cross n=24 requests share a domain
    for t, (fd, p, f, A) in bufs.items():
        P = host(p)
        lu = spla.splu(A.tocsc())
        for r in range(f.shape[0]):
            assert infos[t][r]["status"] == B.FPG_OK and infos[t][r]["residual"] <= 1e-12
            assert rel(P[r], lu.solve(f[r])) < 1e-9
    batch.close()


def test_coalescing_eviction_and_budget(lib):
    from paper_2509_23180_gb300 import binding as B
    n = 32
    d1 = B.make_desc("cross", n, 0.0, nrhs=3)
    need = B.workspace_bytes(B.make_desc("cross", n, 0.0, nrhs=8)) + 8 * 8 * B.unknowns(d1)
    # room for one domain of 8 slots, not two
    batch = B.Batch(int(need * 1.5), slots=8, max_domains=4)
    f = dev(W.rhs_batch("cross", n, [0, 1, 2], kind="fourier"))
    ps = [torch.zeros_like(f) for _ in range(3)]
    live = {batch.admit(d1, f, ps[0]): 3}
    live[batch.admit(d1, f, ps[1])] = 3
    live[batch.admit(B.make_desc("cross", n, 0.0, nrhs=2), f[:2], ps[2][:2])] = 2
    assert batch.stats()["queued"] == 3
    batch.step()  # the idle domain takes all three (3 + 3 + 2 = 8 slots) in one batch
    st = batch.stats()
    assert st["queued"] == 0 and st["busy"] == 1
    run(batch, live)
    assert torch.equal(ps[0], ps[1]) and torch.equal(ps[0][:2], ps[2][:2])
    # another key does not fit beside the idle domain: the idle one is evicted
    d2 = B.make_desc("cross", n, -10.0, nrhs=1)
    t = batch.admit(d2, f[:1], ps[0][:1])
    assert batch.stats()["evicted"] == 1
    run(batch, {t: 1})
    # a key larger than the whole pool is refused and nothing is queued
    with pytest.raises(B.FpgError) as e:
        batch.admit(B.make_desc("cross", 512, 0.0, nrhs=1), f[:1], ps[0][:1])
    assert e.value.status == B.FPG_EBUDGET
    with pytest.raises(B.FpgError) as e:
        batch.poll(123456, 1)
    assert e.value.status == B.FPG_EINVAL
    batch.close()


def test_native_serving_loop(lib):
    from paper_2509_23180_gb300 import serve
    reqs = W.serving_requests(40, 400.0, seed=3)
    res, st = serve.serve_native(reqs, pool_bytes=16e9, realtime=True)
    summ = serve.summarize(res, max(r.end_s for r in res))
    assert summ["all_converged"] and summ["residual_max"] <= 1e-10
    assert st["open_tickets"] == 0 and st["created"] >= 1
