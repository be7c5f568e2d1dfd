"""Request serving on one GPU: continuous batching of solves of mixed geometry
and size, admitted against an HBM budget.

Requests (geometry, n, kappa, 1..slot_rhs right-hand sides) arrive over time.
The server keeps device-resident domains -- workspaces with the tables, Krylov
basis and Hessenberg state of Alg. "fft_dd_solver" -- keyed by (geometry, n,
kappa), each with `slot_rhs` right-hand-side slots and its own CUDA stream.  A
request is admitted as soon as a worker is free and the bytes of all live
domains fit the budget (idle domains of other keys are evicted, least recently
used first, to make room).  Up to `max_inflight` requests run at once, each on
its domain's stream from its own host thread (the library call releases the
GIL), so the kernels of different requests overlap on the device while new
requests keep arriving.  Unused slots of a domain carry a zero right-hand side,
which the solver marks converged before the first Arnoldi step.

Everything on the device goes through the C ABI (paper_2509_23180_gb300.binding);
torch provides the workspaces, the streams and the device-side input generation.
"""
from __future__ import annotations

import threading
import time
from collections import OrderedDict
from concurrent.futures import ThreadPoolExecutor
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
        self._idle = OrderedDict()   # key -> list of idle (Domain, stream, p-buffer)
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
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(stream):
            dom = B.Domain(self._desc(key), stream=stream, device=self.device)
            p = torch.zeros((self.slot_rhs, dom.N), dtype=torch.float64, device=self.device)
        self.created += 1
        return dom, stream, p

    def _release(self, key, entry):
        with self._lock:
            self._idle.setdefault(key, []).append(entry)
            self._idle.move_to_end(key)
            self._lock.notify_all()

    # -- one request -----------------------------------------------------
    def solve_request(self, req: dict, t0: float, arrival_s: float | None = None) -> Result:
        """Solve one request (on the calling thread); times are seconds after t0;
        arrival_s overrides the request's own arrival time."""
        import workloads as W
        torch = self.torch
        key = (req["geometry"], int(req["n"]), float(req["kappa"]))
        nr = int(req["nrhs"])
        if nr < 1 or nr > self.slot_rhs:
            raise ValueError(f"request {req['id']}: nrhs {nr} outside 1..{self.slot_rhs}")
        entry = self._acquire(key)
        dom, stream, p = entry
        start = time.perf_counter() - t0
        try:
            with torch.cuda.stream(stream):
                f = torch.zeros((self.slot_rhs, dom.N), dtype=torch.float64, device=self.device)
                for r in range(nr):
                    f[r] = W.fourier_rhs_torch(key[0], key[1], int(req["seed"]) * 16 + r, device=self.device)
                dom.set_rhs(f)
                st, info = dom.solve(p, check=False)
                sol = p[:nr].to("cpu", non_blocking=False) if self.keep else None
            end = time.perf_counter() - t0
        finally:
            self._release(key, entry)
        arr = float(req["arrival_s"]) if arrival_s is None else arrival_s
        return Result(id=int(req["id"]), arrival_s=arr, start_s=start, end_s=end, nrhs=nr,
                      iterations=[i["iterations"] for i in info[:nr]],
                      residuals=[i["residual"] for i in info[:nr]],
                      status=max([i["status"] for i in info[:nr]] or [0]), solution=sol)

    # -- a stream of requests ---------------------------------------------
    def serve(self, requests, realtime: bool = True):
        """Run a request stream: each request is submitted at its arrival time
        (realtime=True), or all of them at time 0 (realtime=False, latencies then
        count from the start of the run); returns the results in request order."""
        pool = ThreadPoolExecutor(max_workers=self.max_inflight)
        t0 = time.perf_counter()
        futs = []
        for req in requests:
            if realtime:
                delay = float(req["arrival_s"]) - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                futs.append(pool.submit(self.solve_request, req, t0))
            else:
                futs.append(pool.submit(self.solve_request, req, t0, 0.0))
        results = [f.result() for f in futs]
        pool.shutdown()
        return results

    def close(self):
        with self._lock:
            for lst in self._idle.values():
                for d, _, p in lst:
                    d.close()
            self._idle.clear()
            self._bytes = 0.0


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
            "all_converged": all(r.status == B.FPG_OK for r in results)}
