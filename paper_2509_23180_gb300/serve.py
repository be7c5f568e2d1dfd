"""Request serving on one GPU: continuous batching of solves of mixed geometry
and size, admitted against an HBM budget.

serve_native() drives the library's batch runtime (fpg_batch_*: queues per
descriptor, resident domains on their own streams, a pool allocator with
eviction) from one host thread, with a producer thread playing the clients;
summarize() reports throughput and latency of a served stream.

Everything on the device goes through the C ABI (paper_2509_23180_gb300.binding);
torch provides the workspaces, the streams and the device-side input generation.
"""
from __future__ import annotations

import threading
import time
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


def serve_native(requests, pool_bytes: float = 120e9, slot_rhs: int = 8, restart: int = 40, rtol: float = 1e-10,
                 precond_precision: int = 32, max_domains: int = 64, max_per_key: int = 2, max_busy: int = 8,
                 realtime: bool = True, device: str = "cuda", io_bytes: float = 32e9,
                 keep_solutions: bool = False, deadline_s: float | None = None):
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
    keeps its buffers and is admitted first when room frees.  With
    keep_solutions, each result carries its solution (a host tensor).  With
    deadline_s, no request is admitted after that many seconds: the ones admitted
    finish, the rest are left out and counted in stats["unserved"].  Returns
    (results of the served requests in request order, stats)."""
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
            status=max([i["status"] for i in info] or [0]), key=(r["geometry"], int(r["n"]), float(r["kappa"])),
            solution=p.cpu() if keep_solutions else None)
        del live[t]
        io_live -= nb
        return True

    th = threading.Thread(target=producer, daemon=True)
    th.start()
    produced_all = False
    past_deadline = False
    try:
        while not produced_all or live or pending or head is not None:
            progressed = False
            if deadline_s is not None and not past_deadline and time.perf_counter() - t0 > deadline_s:
                # admit nothing more: drop the backlog, let the admitted requests finish
                past_deadline = True
                stop.set()
                produced_all = True
                pending.clear()
                if head is not None:
                    io_live -= head[4]
                    head = None
            while not past_deadline:  # arrivals: host side only
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
    served = [results[int(r["id"])] for r in requests if int(r["id"]) in results]
    stats["unserved"] = len(requests) - len(served)
    return served, stats


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
