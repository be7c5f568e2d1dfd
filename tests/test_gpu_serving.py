"""Serving: continuous batching of mixed requests under an HBM budget, through
the library's batch runtime (fpg_batch_*) driven by serve.serve_native (GPU).

Each result is the same, bit for bit, alone and in the mix (requests of mixed
geometry, size and kappa coalesced into shared domains, running concurrently
on the device); served answers match the oracle; a pool that holds few domains
forces eviction and re-creation; a request larger than the pool is refused.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _requests(count=10, seed=11, sizes=(16, 24, 31), first_id=0):
    rng = np.random.default_rng(seed)
    geoms = ("L", "T", "cross")
    return [{"id": first_id + i, "arrival_s": 0.0, "geometry": geoms[i % 3], "n": int(rng.choice(sizes)),
             "nrhs": int(rng.integers(1, 4)), "kappa": (0.0, -10.0)[i % 2], "seed": 100 + i}
            for i in range(count)]


def _serve(reqs, pool=4e9, **kw):
    from paper_2509_23180_gb300 import serve
    return serve.serve_native(reqs, pool_bytes=pool, slot_rhs=3, restart=30, rtol=1e-11, precond_precision=64,
                              realtime=False, keep_solutions=True, **kw)


def test_results_same_alone_and_in_the_mix(lib):
    """Each request's solution is the same when it is served alone as when it is
    served with nine others (mixed geometry, size, kappa; coalesced into shared
    domains, several domains busy at once)."""
    reqs = _requests()
    res_mix, _ = _serve(reqs, max_busy=4)
    for req, r in zip(reqs, res_mix):
        a = _serve([req], max_busy=1)[0][0]
        assert r.status == 0 and a.status == 0
        assert np.array_equal(r.solution.numpy(), a.solution.numpy()), req
        assert max(r.residuals) <= 1e-11
    # and the served answers are the oracle's
    req, r = reqs[3], res_mix[3]
    K = O.assemble(req["geometry"], req["n"], req["kappa"])
    for k in range(req["nrhs"]):
        f = W.fourier_rhs(req["geometry"], req["n"], req["seed"] * 16 + k)
        ref = D.solve(K, f)
        assert np.abs(r.solution.numpy()[k] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_small_pool_evicts_and_recreates(lib):
    """A pool that holds about two domains, 30 requests over many keys: idle
    domains are evicted and re-created, every request converges, and sampled
    results equal their results alone."""
    from paper_2509_23180_gb300 import binding as B
    reqs = _requests(30, seed=5, sizes=(8, 12, 16, 20))
    need = max(B.workspace_bytes(B.make_desc(q["geometry"], q["n"], q["kappa"], nrhs=3, restart=30))
               + 8 * 3 * B.unknowns(B.make_desc(q["geometry"], q["n"], q["kappa"], nrhs=3)) for q in reqs)
    res, st = _serve(reqs, pool=2.5 * need, max_busy=2)
    assert st["evicted"] >= 1 and st["created"] > len({(q["geometry"], q["n"], q["kappa"]) for q in reqs}) - 1
    assert all(r.status == 0 for r in res)
    for req, r in list(zip(reqs, res))[::7]:
        a = _serve([req], max_busy=1)[0][0]
        assert np.array_equal(r.solution.numpy(), a.solution.numpy()), req


def test_request_over_budget_is_refused(lib):
    from paper_2509_23180_gb300 import binding as B
    with pytest.raises(B.FpgError) as e:
        _serve([{"id": 0, "arrival_s": 0.0, "geometry": "cross", "n": 64, "nrhs": 1, "kappa": 0.0, "seed": 1}],
               pool=1e6)
    assert e.value.status == B.FPG_EBUDGET


def test_set_stream_keeps_the_answer(lib):
    from paper_2509_23180_gb300 import binding as B
    n = 24
    f = torch.as_tensor(W.rhs_batch("cross", n, [0, 1], kind="fourier"), device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    d = B.Domain(B.make_desc("cross", n, 0.0, nrhs=2, restart=10, rtol=1e-11), stream=s1)
    p1 = torch.zeros_like(f)
    d.set_rhs(f)
    assert d.solve(p1)[0] == B.FPG_OK
    d.set_stream(s2)
    p2 = torch.zeros_like(f)
    d.set_rhs(f)
    assert d.solve(p2)[0] == B.FPG_OK
    d.close()
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
