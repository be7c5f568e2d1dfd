"""Request serving on one GPU: continuous batching of solves of mixed geometry
and size, admitted against an HBM budget.

Two request loops share the Result type and summarize():
  serve_native()  -- the library's batch runtime (fpg_batch_*: queues per
                     descriptor, resident domains on their own streams, pool
                     allocator with eviction) driven from one host thread, with a
                     producer thread playing the clients;
  Server.serve()  -- worker threads that each run whole solves on domains they
                     take from a Python-side pool (described below).

Requests (geometry, n, kappa, 1..slot_rhs right-hand sides) arrive over time.
The server keeps device-resident domains -- workspaces with the tables, Krylov
basis and Hessenberg state of Alg. "fft_dd_solver" -- keyed by (geometry, n,
kappa), each with `slot_rhs` right-hand-side slots.  A request is admitted as
soon as a worker is free and the bytes of all live domains fit the budget (idle
domains of other keys are evicted, least recently used first, to make room).
Up to `max_inflight` workers run at once, each from its own host thread (the
library call releases the GIL) on that worker's own CUDA stream -- the domain
is moved onto it with fpg_set_stream -- so the kernels of different requests
overlap on the device while new requests keep arriving.  A free worker takes
the oldest pending request together with later pending requests of the same
key whose right-hand sides still fit the domain's slots, and solves them in
one batch (each right-hand side is solved independently, so a result does not
depend on its slot or its batch mates).  Streams belong to
workers, not domains: torch hands out pooled streams, and a domain created per
stream would, after enough creations, share a stream with a domain that is
running in another thread.  Unused slots of a domain carry a zero right-hand side,
which the solver marks converged before the first Arnoldi step.

Everything on the device goes through the C ABI (paper_2509_23180_gb300.binding);
torch provides the workspaces, the streams and the device-side input generation.
"""
from __future__ import annotations

import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field

from . import binding as B


@dataclass
class Result:
    id: int
    arrival_s: float
    start_s: float
    end_s: float
    nrhs: int
    iterations: list = field(default_factory=list)
    residuals: list = field(default_factory=list)
    status: int = 0
    solution: object = None  # host tensor (nrhs, unknowns) when keep_solutions
    key: tuple = ()          # (geometry, n, kappa)

    @property
    def latency_s(self) -> float:
        return self.end_s - self.arrival_s


class Server:
    def __init__(self, budget_bytes: float = 120e9, max_inflight: int = 8, slot_rhs: int = 8, restart: int = 40,
                 rtol: float = 1e-10, precond_precision: int = 32, keep_solutions: bool = False, device: str = "cuda"):
        import torch
        self.torch = torch
        self.budget = float(budget_bytes)
        self.max_inflight = max_inflight
        self.slot_rhs = slot_rhs
        self.restart = restart
        self.rtol = rtol
        self.precision = precond_precision
        self.keep = keep_solutions
        self.device = device
        self._lock = threading.Condition()
        # one stream per worker thread, created up front (distinct pooled streams)
        self._streams = [torch.cuda.Stream(device=device) for _ in range(max_inflight)]
        self._next_stream = 0
        self._tls = threading.local()
        self._idle = OrderedDict()   # key -> list of idle (Domain, None, p-buffer)
        self._bytes = 0.0            # workspace bytes of all live domains
        self._live = 0
        self.created = 0
        self.evicted = 0
        self.peak_bytes = 0.0

    # -- domains ---------------------------------------------------------
    def _desc(self, key):
        geom, n, kappa = key
        return B.make_desc(geom, n, kappa, nrhs=self.slot_rhs, restart=self.restart, rtol=self.rtol,
                           precond_precision=self.precision)

    def domain_bytes(self, key) -> int:
        """Device bytes a domain of this key occupies (workspace + solution buffer)."""
        d = self._desc(key)
        return B.workspace_bytes(d) + 8 * self.slot_rhs * B.unknowns(d)

    def _acquire(self, key):
        need = self.domain_bytes(key)
        if need > self.budget:
            raise B.FpgError(B.FPG_EBUDGET, "admission", f"one domain of {key} needs {need} bytes > budget")
        with self._lock:
            while True:
                lst = self._idle.get(key)
                if lst:
                    entry = lst.pop()
                    if not lst:
                        del self._idle[key]
                    return entry
                # make room: evict idle domains of other keys, oldest first
                while self._bytes + need > self.budget and self._idle:
                    k_old, lst_old = next(iter(self._idle.items()))
                    d_old, _, p_old = lst_old.pop()
                    if not lst_old:
                        del self._idle[k_old]
                    self._bytes -= self.domain_bytes(k_old)
                    self._live -= 1
                    self.evicted += 1
                    d_old.close()
                    del p_old
                if self._bytes + need <= self.budget:
                    self._bytes += need
                    self._live += 1
                    self.peak_bytes = max(self.peak_bytes, self._bytes)
                    break
                self._lock.wait()  # every other domain is busy: wait for a release
        torch = self.torch
        stream = self._worker_stream()
        with torch.cuda.stream(stream):
            dom = B.Domain(self._desc(key), stream=stream, device=self.device)
            p = torch.zeros((self.slot_rhs, dom.N), dtype=torch.float64, device=self.device)
        self.created += 1
        return dom, None, p

    def _worker_stream(self):
        s = getattr(self._tls, "stream", None)
        if s is None:
            with self._lock:
                s = self._streams[self._next_stream % len(self._streams)]
                self._next_stream += 1
            self._tls.stream = s
        return s

    def _release(self, key, entry):
        with self._lock:
            self._idle.setdefault(key, []).append(entry)
            self._idle.move_to_end(key)
            self._lock.notify_all()

    # -- one solve: one or more requests of the same key --------------------
    def solve_batch(self, reqs, t0: float, arrival_override: float | None = None):
        """Solve requests of one key together on one domain (their right-hand
        sides fill consecutive slots; on the calling thread); times are seconds
        after t0.  Returns one Result per request."""
        import workloads as W
        torch = self.torch
        key = (reqs[0]["geometry"], int(reqs[0]["n"]), float(reqs[0]["kappa"]))
        nrs = [int(r["nrhs"]) for r in reqs]
        for r, nr in zip(reqs, nrs):
            if nr < 1 or nr > self.slot_rhs:
                raise ValueError(f"request {r['id']}: nrhs {nr} outside 1..{self.slot_rhs}")
            if (r["geometry"], int(r["n"]), float(r["kappa"])) != key:
                raise ValueError("solve_batch: requests of different keys")
        if sum(nrs) > self.slot_rhs:
            raise ValueError("solve_batch: more right-hand sides than slots")
        entry = self._acquire(key)
        dom, _, p = entry
        stream = self._worker_stream()
        if dom.stream is not stream:
            dom.set_stream(stream)  # the previous user's work finished before its release
        start = time.perf_counter() - t0
        try:
            with torch.cuda.stream(stream):
                f = torch.zeros((self.slot_rhs, dom.N), dtype=torch.float64, device=self.device)
                slot = 0
                for r, nr in zip(reqs, nrs):
                    for i in range(nr):
                        f[slot] = W.fourier_rhs_torch(key[0], key[1], int(r["seed"]) * 16 + i, device=self.device)
                        slot += 1
                dom.set_rhs(f)
                st, info = dom.solve(p, check=False)
                sol = p[:slot].to("cpu", non_blocking=False) if self.keep else None
            end = time.perf_counter() - t0
        finally:
            self._release(key, entry)
        out, s0 = [], 0
        for r, nr in zip(reqs, nrs):
            arr = float(r["arrival_s"]) if arrival_override is None else arrival_override
            inf = info[s0:s0 + nr]
            out.append(Result(id=int(r["id"]), arrival_s=arr, start_s=start, end_s=end, nrhs=nr,
                              iterations=[i["iterations"] for i in inf], residuals=[i["residual"] for i in inf],
                              status=max([i["status"] for i in inf] or [0]),
                              solution=sol[s0:s0 + nr] if sol is not None else None, key=key))
            s0 += nr
        return out

    def solve_request(self, req: dict, t0: float, arrival_s: float | None = None) -> Result:
        """Solve one request alone (on the calling thread)."""
        return self.solve_batch([req], t0, arrival_s)[0]

    # -- a stream of requests ---------------------------------------------
    def serve(self, requests, realtime: bool = True):
        """Run a request stream with continuous batching: requests enter a
        pending queue at their arrival time (realtime=True; else all at time 0,
        latencies then count from the start of the run).  Each of max_inflight
        workers takes the oldest pending request plus the next pending requests
        of the same (geometry, n, kappa) while their right-hand sides fit the
        domain's slots, and solves them together; requests that arrive while
        others are on the GPU join the queue and go out with the next free
        worker.  Returns the results in request order."""
        t0 = time.perf_counter()
        pending = []              # arrived, not yet taken (FIFO)
        cv = threading.Condition()
        state = {"closed": False, "error": None}
        results = {}
        self.coalesced = 0

        def key_of(r):
            return (r["geometry"], int(r["n"]), float(r["kappa"]))

        def worker():
            while True:
                with cv:
                    while not pending and not state["closed"] and state["error"] is None:
                        cv.wait()
                    if state["error"] is not None or (not pending and state["closed"]):
                        return
                    head = pending.pop(0)
                    batch, room, k = [head], self.slot_rhs - int(head["nrhs"]), key_of(head)
                    i = 0
                    while i < len(pending) and room > 0:
                        r = pending[i]
                        if key_of(r) == k and int(r["nrhs"]) <= room:
                            batch.append(pending.pop(i))
                            room -= int(r["nrhs"])
                        else:
                            i += 1
                    self.coalesced += len(batch) - 1
                try:
                    res = self.solve_batch(batch, t0, None if realtime else 0.0)
                except BaseException as e:  # stop the stream; re-raised below
                    with cv:
                        state["error"] = e
                        cv.notify_all()
                    return
                with cv:
                    for r in res:
                        results[r.id] = r

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.max_inflight)]
        for th in threads:
            th.start()
        for req in requests:
            if state["error"] is not None:
                break
            if realtime:
                delay = float(req["arrival_s"]) - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            with cv:
                pending.append(req)
                cv.notify()
        with cv:
            state["closed"] = True
            cv.notify_all()
        for th in threads:
            th.join()
        if state["error"] is not None:
            raise state["error"]
        return [results[int(r["id"])] for r in requests]

    def close(self):
        with self._lock:
            for lst in self._idle.values():
                for d, _, p in lst:
                    d.close()
            self._idle.clear()
            self._bytes = 0.0


def serve_native(requests, pool_bytes: float = 120e9, slot_rhs: int = 8, restart: int = 40, rtol: float = 1e-10,
                 precond_precision: int = 32, max_domains: int = 64, max_per_key: int = 2, max_busy: int = 8,
                 realtime: bool = True, device: str = "cuda", io_bytes: float = 32e9):
    """The request stream through the library's batch runtime (fpg_batch_*).
    A producer thread plays the clients: at each request's arrival time it hands
    the request (its descriptor and seed, host side) to the driver thread.  The
    driver admits requests in arrival order: it builds a request's right-hand
    sides and solution buffer on the device only when it admits it, and only
    while the buffers of admitted, unfinished requests stay within `io_bytes`
    (a backlog waits on the host, not in HBM).  The runtime queues an admitted
    request with the other requests of its (geometry, n, kappa) for the next
    batch of a resident domain and evicts idle domains when the pool is short;
    the driver steps it -- the runtime never waits on the device -- and collects
    the tickets it reports finished.  A request refused for lack of idle room
    keeps its buffers and is admitted first when room frees.  Returns (results
    in request order, stats)."""
    import queue
    from collections import deque

    import torch

    import workloads as W
    batch = B.Batch(int(pool_bytes), slots=slot_rhs, max_domains=max_domains, max_per_key=max_per_key,
                    max_busy=max_busy, device=device)
    order = sorted(range(len(requests)), key=lambda i: float(requests[i]["arrival_s"]))
    ready = queue.Queue()
    live = {}          # ticket -> (request, f, p, admit time, buffer bytes)
    pending = deque()  # arrived, not yet built on the device (arrival order)
    head = None        # built, refused for room: admitted first
    results = {}
    io_live = 0
    gen = torch.cuda.Stream(device=device)
    t0 = time.perf_counter()
    stop = threading.Event()
    failed = []        # the producer's exception, re-raised by the driver thread

    def producer():
        try:
            for i in order:
                if stop.is_set():
                    return
                r = requests[i]
                if realtime:
                    delay = float(r["arrival_s"]) - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                ready.put(r)
        except BaseException as e:
            failed.append(e)
        finally:
            ready.put(None)

    def desc_of(r):
        return B.make_desc(r["geometry"], int(r["n"]), float(r["kappa"]), nrhs=int(r["nrhs"]), restart=restart,
                           rtol=rtol, precond_precision=precond_precision)

    def buffer_bytes(r):
        return 2 * 8 * int(r["nrhs"]) * B.unknowns(desc_of(r))

    def build(r):
        geom, n, nr = r["geometry"], int(r["n"]), int(r["nrhs"])
        with torch.cuda.stream(gen):
            f = torch.stack([W.fourier_rhs_torch(geom, n, int(r["seed"]) * 16 + j, device=device)
                             for j in range(nr)])
            p = torch.empty_like(f)
        gen.synchronize()  # f final before the runtime copies it
        return (r, desc_of(r), f, p, buffer_bytes(r))

    def key_bytes(desc):
        full = B.make_desc(desc.geometry, desc.n, desc.kappa, nrhs=slot_rhs, restart=restart, rtol=rtol,
                           precond_precision=precond_precision)
        return B.workspace_bytes(full) + 8 * slot_rhs * B.unknowns(full)

    def try_admit(entry):
        r, desc, f, p, nb = entry
        try:
            live[batch.admit(desc, f, p)] = (r, f, p, time.perf_counter() - t0, nb)
            return True
        except B.FpgError as e:
            if e.status != B.FPG_EBUDGET or key_bytes(desc) > pool_bytes:
                raise
            return False

    def collect(t):
        nonlocal io_live
        r, f, p, t_adm, nb = live[t]
        info = batch.poll(t, int(r["nrhs"]))
        if info is None:
            return False
        results[int(r["id"])] = Result(
            id=int(r["id"]), arrival_s=float(r["arrival_s"]) if realtime else 0.0, start_s=t_adm,
            end_s=time.perf_counter() - t0, nrhs=int(r["nrhs"]),
            iterations=[i["iterations"] for i in info], residuals=[i["residual"] for i in info],
            status=max([i["status"] for i in info] or [0]), key=(r["geometry"], int(r["n"]), float(r["kappa"])))
        del live[t]
        io_live -= nb
        return True

    th = threading.Thread(target=producer, daemon=True)
    th.start()
    produced_all = False
    try:
        while not produced_all or live or pending or head is not None:
            progressed = False
            while True:  # arrivals: host side only
                try:
                    r = ready.get_nowait()
                except queue.Empty:
                    break
                if r is None:
                    if failed:
                        raise RuntimeError("request producer failed") from failed[0]
                    produced_all = True
                    break
                pending.append(r)
                progressed = True
            if head is not None and try_admit(head):
                head = None
                progressed = True
            while head is None and pending:
                nb = buffer_bytes(pending[0])
                if (live or io_live) and io_live + nb > io_bytes:
                    break  # request buffers at their cap: the backlog waits on the host
                entry = build(pending.popleft())
                io_live += nb
                progressed = True
                if not try_admit(entry):
                    head = entry
            finished = batch.step()
            for t in finished:
                progressed |= collect(t)
            if len(finished) >= batch.report_cap:  # more finished than reported: poll the rest
                for t in list(live):
                    collect(t)
            if not progressed:
                time.sleep(5e-5)
        stats = batch.stats()
    finally:
        stop.set()
        th.join()
        batch.close()
    return [results[int(r["id"])] for r in requests], stats


def summarize(results, wall_s: float) -> dict:
    """Throughput and latency of a served stream."""
    import numpy as np
    lat = np.array([r.latency_s for r in results]) * 1e3
    solves = sum(r.nrhs for r in results)
    res = [x for r in results for x in r.residuals]
    return {"requests": len(results), "solves": solves, "wall_s": wall_s,
            "solves_per_s": solves / wall_s if wall_s > 0 else None,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "residual_max": max(res) if res else None,
            "all_converged": all(r.status == B.FPG_OK for r in results),
            "failures": [{"id": r.id, "key": list(r.key), "nrhs": r.nrhs, "status": r.status,
                          "iterations": r.iterations, "residuals": r.residuals}
                         for r in results if r.status != B.FPG_OK][:12]}
