"""Serving: continuous batching of mixed requests under an HBM budget (GPU)."""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import operator as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _requests():
    rng = np.random.default_rng(11)
    geoms = ("L", "T", "cross")
    reqs = []
    for i in range(10):
        reqs.append({"id": i, "arrival_s": 0.0, "geometry": geoms[i % 3], "n": int(rng.choice([16, 24, 31])),
                     "nrhs": int(rng.integers(1, 4)), "kappa": (0.0, -10.0)[i % 2], "seed": 100 + i})
    return reqs


def test_results_same_alone_and_in_the_mix(lib):
    """Each request's solution is the same when it runs alone as when it runs
    concurrently with nine others (mixed geometry, size, kappa)."""
    from paper_2509_23180_gb300 import serve
    reqs = _requests()
    mix = serve.Server(budget_bytes=4e9, max_inflight=4, slot_rhs=3, restart=30, rtol=1e-11,
                       precond_precision=64, keep_solutions=True)
    res_mix = mix.serve(reqs, realtime=False)
    mix.close()
    for req, r in zip(reqs, res_mix):
        alone = serve.Server(budget_bytes=4e9, max_inflight=1, slot_rhs=3, restart=30, rtol=1e-11,
                             precond_precision=64, keep_solutions=True)
        a = alone.serve([req], realtime=False)[0]
        alone.close()
        assert r.status == 0 and a.status == 0
        assert np.array_equal(r.solution.numpy(), a.solution.numpy()), req
        assert max(r.residuals) <= 1e-11
    # and the served answers are the oracle's
    req, r = reqs[3], res_mix[3]
    K = O.assemble(req["geometry"], req["n"], req["kappa"])
    for k in range(req["nrhs"]):
        f = W.fourier_rhs(req["geometry"], req["n"], req["seed"] * 16 + k)
        ref = D.solve(K, f)
        assert np.linalg.norm(r.solution.numpy()[k] - ref) / np.linalg.norm(ref) < 1e-9


def test_admission_respects_the_budget(lib):
    """With room for one domain only, requests of different keys still all
    complete: idle domains are evicted and the live bytes never exceed the budget."""
    from paper_2509_23180_gb300 import serve
    reqs = _requests()[:5]
    probe = serve.Server(slot_rhs=3, restart=30)
    need = max(probe.domain_bytes((r["geometry"], r["n"], r["kappa"])) for r in reqs)
    s = serve.Server(budget_bytes=1.5 * need, max_inflight=3, slot_rhs=3, restart=30, rtol=1e-10,
                     precond_precision=32)
    res = s.serve(reqs, realtime=False)
    assert all(r.status == 0 for r in res)
    assert s.peak_bytes <= 1.5 * need
    assert s.evicted >= 1
    s.close()
    summary = serve.summarize(res, max(r.end_s for r in res))
    assert summary["all_converged"] and summary["solves"] == sum(r["nrhs"] for r in reqs)


def test_request_over_budget_is_refused(lib):
    from paper_2509_23180_gb300 import binding as B
    from paper_2509_23180_gb300 import serve
    s = serve.Server(budget_bytes=1e6, max_inflight=1, slot_rhs=2)
    with pytest.raises(B.FpgError) as e:
        s.serve([{"id": 0, "arrival_s": 0.0, "geometry": "cross", "n": 64, "nrhs": 1, "kappa": 0.0, "seed": 1}],
                realtime=False)
    assert e.value.status == B.FPG_EBUDGET


def test_many_domain_creations_with_graphs(lib):
    """More domain creations than torch's pool of streams (32), under a budget
    that forces eviction, with graph capture on and 8 concurrent workers: every
    request converges and matches its result alone (workers own the streams, so
    a capture never shares its stream with another running domain)."""
    from paper_2509_23180_gb300 import serve
    rng = np.random.default_rng(5)
    geoms = ("L", "T", "cross")
    reqs = [{"id": i, "arrival_s": 0.0, "geometry": geoms[i % 3], "n": int(rng.choice([8, 12, 16, 20])),
             "nrhs": int(rng.integers(1, 3)), "kappa": (0.0, -10.0)[(i // 3) % 2], "seed": 300 + i}
            for i in range(72)]
    probe = serve.Server(slot_rhs=2, restart=20)
    need = max(probe.domain_bytes((r["geometry"], r["n"], r["kappa"])) for r in reqs)
    s = serve.Server(budget_bytes=9 * need, max_inflight=8, slot_rhs=2, restart=20, rtol=1e-11,
                     precond_precision=64, keep_solutions=True)
    res = s.serve(reqs, realtime=False)
    created = s.created
    s.close()
    assert created > 24
    assert all(r.status == 0 for r in res)
    for req, r in list(zip(reqs, res))[::9]:
        alone = serve.Server(budget_bytes=4e9, max_inflight=1, slot_rhs=2, restart=20, rtol=1e-11,
                             precond_precision=64, keep_solutions=True)
        a = alone.serve([req], realtime=False)[0]
        alone.close()
        assert np.array_equal(r.solution.numpy(), a.solution.numpy()), req


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
