"""Host logic of serve_native (CPU only): the request loop around the batch
runtime, driven against a fake runtime that keeps the same contract as
fpg_batch_* (admit refuses with FPG_EBUDGET when the pool is short, step
reports the tickets that finished, poll hands each result out once).

What the loop must guarantee whatever the device does:
  * every request gets exactly one result, in request order;
  * a request refused for lack of room waits and is admitted before any later
    arrival (first come, first admitted), once room frees;
  * a request that could never fit the pool is an error, not an endless wait;
  * more finished tickets than one step reports are still all collected;
  * the device buffers of admitted, unfinished requests stay within the loop's
    cap: a backlog waits on the host;
  * a failure while preparing a request ends the loop with that error (and the
    runtime is closed), instead of a missing result.
"""
import contextlib

import pytest

torch = pytest.importorskip("torch")

from paper_2509_23180_gb300 import binding as B
from paper_2509_23180_gb300 import build as Bd
from paper_2509_23180_gb300 import serve as S
import workloads as W

pytestmark = pytest.mark.timeout(120)


@pytest.fixture(scope="module", autouse=True)
def library():
    Bd.build()  # serve_native sizes domains through fpg_workspace_bytes / fpg_unknowns (host only)
    return B.load()


class FakeBatch:
    """A pool of `pool_bytes`; each admitted request holds its key's bytes
    until it finishes, `latency` steps after admission."""

    log = None
    report_cap = 256

    def __init__(self, pool_bytes, slots=8, max_domains=64, max_per_key=2, max_busy=0, device="cuda",
                 latency=3, report_cap=256, finish_every=1):
        self.pool_bytes, self.slots, self.latency, self.report_cap = pool_bytes, slots, latency, report_cap
        self.finish_every = finish_every  # tickets finish only on every finish_every-th step
        self.truncated = 0
        self.used = 0
        self.next = 1
        self.running = {}   # ticket -> [steps left, bytes, nrhs]
        self.done = {}      # ticket -> nrhs
        self.admitted = []  # (ticket, n, nrhs) in admission order
        self.steps = 0
        self.refused = 0
        FakeBatch.log = self

    def key_bytes(self, desc):
        full = B.make_desc(desc.geometry, desc.n, desc.kappa, nrhs=self.slots, restart=desc.restart,
                           rtol=desc.rtol, precond_precision=desc.precond_precision)
        return B.workspace_bytes(full) + 8 * self.slots * B.unknowns(full)

    def admit(self, desc, f, p):
        assert 1 <= desc.nrhs <= self.slots and f.shape[0] == desc.nrhs
        need = self.key_bytes(desc)
        if self.used + need > self.pool_bytes:
            self.refused += 1
            raise B.FpgError(B.FPG_EBUDGET, "fpg_batch_admit")
        self.used += need
        t = self.next
        self.next += 1
        self.running[t] = [self.latency, need, desc.nrhs]
        self.io = getattr(self, "io", 0) + 2 * 8 * f.numel()  # f and its solution buffer
        self.io_max = max(getattr(self, "io_max", 0), self.io)
        self.io_of = getattr(self, "io_of", {})
        self.io_of[t] = 2 * 8 * f.numel()
        self.admitted.append((t, desc.n, desc.nrhs))
        return t

    def step(self):
        self.steps += 1
        fin = []
        for t in list(self.running):
            self.running[t][0] -= 1
            if self.running[t][0] <= 0 and self.steps % self.finish_every == 0:
                _, need, nrhs = self.running.pop(t)
                self.used -= need
                self.io -= self.io_of.pop(t)
                self.done[t] = nrhs
                fin.append(t)
        self.truncated += len(fin) > self.report_cap
        return fin[:self.report_cap]

    def poll(self, t, nrhs):
        if t not in self.done:
            return None
        assert self.done.pop(t) == nrhs
        return [{"iterations": 7, "restarts": 0, "status": B.FPG_OK, "residual": 1e-11, "schur_residual": 1e-11}
                for _ in range(nrhs)]

    def stats(self):
        return {"created": 0, "evicted": 0, "steps": self.steps}

    def close(self):
        self.left = len(self.running) + len(self.done)  # tickets neither finished nor collected


class _Stream:
    def __init__(self, device=None):
        pass

    def synchronize(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    def make(**kw):
        monkeypatch.setattr(B, "Batch", lambda *a, **k: FakeBatch(*a, **{**k, **kw}))
        monkeypatch.setattr(torch.cuda, "Stream", _Stream)
        monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
        monkeypatch.setattr(W, "fourier_rhs_torch",
                            lambda g, n, seed, device=None: torch.zeros(W.total_unknowns(g, n), dtype=torch.float64))
    return make


def _requests(count, seed=3, sizes=(16, 32, 64)):
    return W.serving_requests(count, 1e6, seed=seed, sizes=sizes, max_rhs=4)


def _bytes(req, slots=8):
    full = B.make_desc(req["geometry"], req["n"], req["kappa"], nrhs=slots, restart=40, rtol=1e-10,
                       precond_precision=32)
    return B.workspace_bytes(full) + 8 * slots * B.unknowns(full)


def test_every_request_gets_one_result_in_order(fake):
    fake()
    reqs = _requests(40)
    res, stats = S.serve_native(reqs, pool_bytes=1 << 40, realtime=False, device="cpu")
    assert [r.id for r in res] == [r["id"] for r in reqs]
    assert all(r.nrhs == q["nrhs"] and len(r.residuals) == q["nrhs"] for r, q in zip(res, reqs))
    assert all(r.status == B.FPG_OK for r in res)
    assert [a[0] for a in FakeBatch.log.admitted] == sorted(a[0] for a in FakeBatch.log.admitted)
    assert FakeBatch.log.left == 0


def test_refused_requests_wait_and_keep_arrival_order(fake):
    fake(latency=200)  # requests stay resident long enough for later arrivals to find the pool full
    reqs = _requests(30)
    # room for about two of the largest requests at a time: most admissions are refused first
    pool = 2 * max(_bytes(q) for q in reqs) + 1
    res, _ = S.serve_native(reqs, pool_bytes=pool, realtime=False, device="cpu")
    assert [r.id for r in res] == [q["id"] for q in reqs]
    by_arrival = sorted(reqs, key=lambda q: q["arrival_s"])
    assert [(a[1], a[2]) for a in FakeBatch.log.admitted] == [(q["n"], q["nrhs"]) for q in by_arrival]
    assert FakeBatch.log.refused >= 10 and FakeBatch.log.used == 0 and FakeBatch.log.left == 0


def test_request_larger_than_the_pool_is_an_error(fake):
    fake()
    reqs = _requests(5)
    pool = min(_bytes(q) for q in reqs) - 1
    with pytest.raises(B.FpgError) as e:
        S.serve_native(reqs, pool_bytes=pool, realtime=False, device="cpu")
    assert e.value.status == B.FPG_EBUDGET


def test_more_finished_than_one_step_reports(fake):
    fake(report_cap=2, latency=1, finish_every=50)
    reqs = _requests(25)
    res, _ = S.serve_native(reqs, pool_bytes=1 << 40, realtime=False, device="cpu")
    assert len(res) == 25 and all(len(r.iterations) == r.nrhs for r in res)
    assert FakeBatch.log.truncated >= 1 and FakeBatch.log.left == 0


def test_request_buffers_stay_within_their_cap(fake):
    """Arrivals far outpace service (every request arrives at once, each stays a
    while): the loop builds a request's buffers only when it admits it, so the
    buffers in the runtime never exceed the cap, and every request still gets
    its result."""
    fake(latency=40)
    reqs = _requests(40)
    per = [2 * 8 * q["nrhs"] * W.total_unknowns(q["geometry"], q["n"]) for q in reqs]
    cap = 3 * max(per)
    res, _ = S.serve_native(reqs, pool_bytes=1 << 40, realtime=False, device="cpu", io_bytes=cap)
    assert [r.id for r in res] == [q["id"] for q in reqs]
    assert 0 < FakeBatch.log.io_max <= cap and FakeBatch.log.left == 0


def test_a_failing_request_build_fails_the_loop(fake, monkeypatch):
    fake(latency=5)
    calls = []

    def rhs(g, n, seed, device=None):
        calls.append(seed)
        if len(calls) > 12:
            raise ValueError("rhs generation failed")
        return torch.zeros(W.total_unknowns(g, n), dtype=torch.float64)

    monkeypatch.setattr(W, "fourier_rhs_torch", rhs)
    with pytest.raises(ValueError):
        S.serve_native(_requests(20), pool_bytes=1 << 40, realtime=False, device="cpu")
    assert hasattr(FakeBatch.log, "left")  # the runtime was still closed


def test_admission_deadline_serves_a_prefix_and_counts_the_rest(fake):
    """With deadline_s, nothing is admitted once that many seconds have passed:
    the requests admitted before it finish and are reported in request order, the
    others are counted as unserved, and the runtime is left empty."""
    fake(latency=2)
    reqs = _requests(30)
    for i, q in enumerate(reqs):  # arrivals 0, 0.01, ... s apart in real time
        q["arrival_s"] = 0.01 * i
    res, stats = S.serve_native(reqs, pool_bytes=1 << 40, realtime=True, device="cpu", deadline_s=0.12)
    served = [r.id for r in res]
    assert 0 < len(served) < len(reqs)
    assert served == [q["id"] for q in reqs][:len(served)]  # a prefix, in request order
    assert stats["unserved"] == len(reqs) - len(served)
    assert FakeBatch.log.left == 0
    # no deadline: everything
    fake(latency=2)
    res, stats = S.serve_native(reqs, pool_bytes=1 << 40, realtime=False, device="cpu")
    assert len(res) == len(reqs) and stats["unserved"] == 0
