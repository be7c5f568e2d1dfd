"""Benchmark: Poisson solves/s of the FFT-preconditioned Schur-complement GMRES
on the cross domain with 256^2 interior points per block (328,704 unknowns),
kappa in {0, -10}, ten seeded random-Fourier right-hand sides per kappa
(20 solves per step), GMRES(30), global relative residual 1e-10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision 64|32] [--n 256] [--seeds 10]

One JSON line on rank 0.  "value" is device-timed solves/s with the inputs
resident in HBM (CUDA events on the library's stream, L2 flushed before every
step); "e2e" repeats the measurement through fpg_solve_host with pinned host
buffers, the copies inside the timed region.  N > 1 runs independent replicas
(one per GPU, no collective) and reports the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s and HBM GB/s at 1e-10 residual vs plain FP64 GPU; p50/p99 latency"
L2_FLUSH_BYTES = 512 << 20
BAD_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=64, choices=[64, 32])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(args):
    return {"workload": f"cross {args.n}^2 per block, kappa in {{0,-10}}, {args.seeds} fourier RHS per kappa",
            "geometry": "cross", "n": args.n, "unknowns_per_rhs": args.n ** 2 + 4 * args.n * (args.n + 1),
            "kappas": [0.0, -10.0], "rhs_per_kappa": args.seeds, "solves_per_step": 2 * args.seeds,
            "restart": args.restart, "rtol": args.rtol, "precond_precision": args.precision,
            "schur_mode": "reduced", "l2": "flushed before every step (512 MiB write)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle arm
def oracle_step(args, f_by_kappa):
    """The FP64 oracle on the same workload: sparse LU of K, then the solves."""
    from oracle import direct, operator
    t0 = time.perf_counter()
    out = {}
    for kappa, f in f_by_kappa.items():
        K = operator.assemble("cross", args.n, kappa)
        out[kappa] = direct.Factor(K).solve(f)
    return time.perf_counter() - t0, out


def cpu_baseline(args, f_by_kappa, max_seconds=30.0):
    """Oracle timed on the host cores on a bounded sample: the factorisation and
    the solves of the first kappa's right-hand sides (the sample shrinks when a
    solve would exceed the time bound)."""
    from oracle import direct, operator
    kappa = 0.0
    f = f_by_kappa[kappa]
    t0 = time.perf_counter()
    K = operator.assemble("cross", args.n, kappa)
    F = direct.Factor(K)
    cnt = 0
    for r in range(f.shape[0]):
        F.solve(f[r])
        cnt += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": cnt / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"kappa=0: assemble + SuperLU factor of K ({K.shape[0]} unknowns) + {cnt} direct solves, "
                      f"{dt:.1f} s (SuperLU and the assembly run single-threaded)"}


def run_reference(args, rank, world):
    import numpy as np
    import workloads as W
    if rank != 0:
        return
    seeds = list(range(args.seeds))
    f_by_kappa = {k: W.rhs_batch("cross", args.n, seeds, kind="fourier") for k in (0.0, -10.0)}
    times = []
    for s in range(args.warmup + args.steps):
        dt, _ = oracle_step(args, f_by_kappa)
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    val = 2 * args.seeds / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(args),
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": "full step: SuperLU factor of K per kappa + all direct solves, single thread"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def algorithmic_costs(n, iters_per_solve, m):
    """Algorithmic work per solve: bytes and flops of each hot-path step."""
    import math
    nc = n * n
    per_iter_bytes = 0.0
    # average Arnoldi index over the iterations of a solve (restart cycles of m)
    jbar = min(iters_per_solve, m) / 2.0
    fs_bytes = 16.0 * nc                       # a1: read v, write z
    fs_flops = (5.0 * math.log2(n) + 6.0) * nc  # a1: two DST-I (2.5 n log2 n each) + Thomas
    sc_bytes = 16.0 * nc                       # a2: read z, write w
    ar_bytes = (8.0 * (jbar + 1) + 24.0) * nc  # a3: V once, w read/write, v_{j+1} write
    ar_flops = (4.0 * (jbar + 1) + 3.0) * nc   # a3: dot + axpy per basis vector, norm, scale
    per_iter_bytes = fs_bytes + sc_bytes + ar_bytes
    return {"fast_solve_bytes": fs_bytes, "fast_solve_flops": fs_flops, "arnoldi_bytes": ar_bytes,
            "arnoldi_flops": ar_flops, "per_iter_bytes": per_iter_bytes,
            "per_solve_bytes": per_iter_bytes * iters_per_solve}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import workloads as W
    from paper_2509_23180_gb300 import binding as B
    from paper_2509_23180_gb300 import build as Bd

    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
    dev_index = torch.cuda.current_device()
    if not os.path.exists(B.LIB_PATH):
        Bd.build()
    B.load()
    seeds = list(range(args.seeds))
    kappas = (0.0, -10.0)
    f_host = {k: W.rhs_batch("cross", args.n, seeds, kind="fourier") for k in kappas}
    doms, fdev, pdev = {}, {}, {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for k in kappas:
            desc = B.make_desc("cross", args.n, k, nrhs=args.seeds, restart=args.restart, rtol=args.rtol,
                               precond_precision=args.precision)
            doms[k] = B.Domain(desc, stream=stream)
            fdev[k] = torch.as_tensor(f_host[k], device="cuda")
            pdev[k] = torch.zeros_like(fdev[k])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(profile=False):
        infos = []
        for k in kappas:
            doms[k].set_rhs(fdev[k])
            st, info = doms[k].solve(pdev[k], check=False)
            infos.append((st, info))
        return infos

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        for k in kappas:
            doms[k].set_profiling(True)
        launches0 = sum(doms[k].launch_count() for k in kappas)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        step_infos = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev_index) as clk:
            for s in range(args.steps):
                flush.fill_(float(s))
                ev[s][0].record(stream)
                step_infos.append(step())
                ev[s][1].record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        launches = sum(doms[k].launch_count() for k in kappas) - launches0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        phases = {}
        for k in kappas:
            for name, v in doms[k].phase_stats().items():
                ph = phases.setdefault(name, {"launches": 0, "ms": 0.0})
                ph["launches"] += v["launches"]
                ph["ms"] += v["ms"]
            doms[k].set_profiling(False)

    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    solves_per_step = 2 * args.seeds
    value = world * solves_per_step / (ms_per_step * 1e-3)

    # correctness of every timed solve (device residuals)
    resid = [i["residual"] for step_i in step_infos for (_, info) in step_i for i in info]
    iters = [i["iterations"] for step_i in step_infos for (_, info) in step_i for i in info]
    ok = all(st == B.FPG_OK for step_i in step_infos for (st, _) in step_i)

    # e2e: host buffers through fpg_solve_host, copies inside the timed region
    fpin = {k: torch.as_tensor(f_host[k]).pin_memory() for k in kappas}
    ppin = {k: torch.empty_like(fpin[k]).pin_memory() for k in kappas}
    with torch.cuda.stream(stream):
        for k in kappas:  # warm the pinned path once
            doms[k].solve_host(fpin[k], ppin[k])
        torch.cuda.synchronize()
    e2e_total = 0.0
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            ta = time.perf_counter()
            for k in kappas:
                doms[k].solve_host(fpin[k], ppin[k])
            e2e_total += time.perf_counter() - ta
    e2e_val = world * solves_per_step * args.steps / e2e_total
    bytes_h2d = sum(fpin[k].numel() * 8 for k in kappas)

    # roofline of the dominant kernel group, from the in-run phase events
    iters_mean = float(np.mean(iters)) if iters else 0.0
    costs = algorithmic_costs(args.n, iters_mean, args.restart)
    peaks = measured_peaks()
    fp64_peak = B.probe_fma_peak(64)
    fp32_peak = B.probe_fma_peak(32)
    dom_phase = max(("precond", "arnoldi", "schur"), key=lambda p: phases[p]["ms"])
    roof = roofline(dom_phase, phases, costs, args, peaks, fp64_peak, fp32_peak, args.seeds, kappas)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 64 else "f64+f32precond", "data": "synthetic",
        "config": workload(args),
        "hbm_gbs_algorithmic": value / world * costs["per_solve_bytes"] / 1e9,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "per": "step of %d solves" % solves_per_step},
        "iterations_mean": iters_mean, "residual_max": max(resid) if resid else None, "all_converged": ok,
        "phases_ms": {k: round(v["ms"] / args.steps, 4) for k, v in phases.items()},
        "gpu_launches": int(launches),
        "roofline": roof,
        "peaks": {"fp64_fma_tflops_probe": fp64_peak / 1e12, "fp32_fma_tflops_probe": fp32_peak / 1e12,
                  "hbm_gbs_measured": peaks.get("hbm_gbs")},
        "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": bytes_h2d,
                "d2h_bytes_per_step": bytes_h2d},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_variants:
        line["variants"] = variants(args, f_host, stream, flush)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, f_host)
    for k in kappas:
        doms[k].close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def variants(args, f_host, stream, flush):
    """Same workload, other forms of the method (device-timed, L2 flushed)."""
    import torch
    from paper_2509_23180_gb300 import binding as B
    out = {}
    kappas = (0.0, -10.0)
    forms = {"fp32_precond": dict(precond_precision=32, nrhs=args.seeds),
             "fp64_single_rhs": dict(precond_precision=64, nrhs=1)}
    if args.precision == 32:
        forms = {"fp64_plain": dict(precond_precision=64, nrhs=args.seeds)}
    for name, kw in forms.items():
        with torch.cuda.stream(stream):
            doms = {k: B.Domain(B.make_desc("cross", args.n, k, restart=args.restart, rtol=args.rtol, **kw),
                                stream=stream) for k in kappas}
            nr = kw["nrhs"]
            fd = {k: torch.as_tensor(f_host[k], device="cuda") for k in kappas}
            pd = {k: torch.zeros_like(fd[k]) for k in kappas}

            def one_step():
                its = []
                for k in kappas:
                    for s0 in range(0, args.seeds, nr):
                        doms[k].set_rhs(fd[k][s0:s0 + nr])
                        st, info = doms[k].solve(pd[k][s0:s0 + nr], check=False)
                        its += [(st, i) for i in info]
                return its
            one_step()
            torch.cuda.synchronize()
            tot = 0.0
            its = []
            for s in range(max(1, min(args.steps, 3))):
                flush.fill_(float(s))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                its += one_step()
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            nsteps = max(1, min(args.steps, 3))
            out[name] = {"solves_per_s": 2 * args.seeds * nsteps / (tot * 1e-3),
                         "iterations_mean": sum(i["iterations"] for _, i in its) / len(its),
                         "residual_max": max(i["residual"] for _, i in its),
                         "all_converged": all(st == B.FPG_OK for st, _ in its)}
            for k in kappas:
                doms[k].close()
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def roofline(phase, phases, costs, args, peaks, fp64_peak, fp32_peak, nrhs, kappas):
    """Roofline entry for the dominant kernel group: algorithmic work per launch
    over its average device duration (CUDA events inside the timed region)."""
    ph = phases[phase]
    calls = max(1, ph["launches"])
    nc = args.n * args.n
    hbm = peaks.get("hbm_gbs", 6800.0)
    if phase == "precond":
        # 3 launches per application (forward DST, Thomas, inverse DST) over nrhs blocks
        apps = calls / 3.0
        t = ph["ms"] * 1e-3 / apps
        flops = costs["fast_solve_flops"] * nrhs
        byts = (16.0 if args.precision == 64 else 12.0) * nc * nrhs
        if args.precision == 64:
            ach = flops / t
            return {"kernel": "fast_solve (forward DST, Thomas, inverse DST; per application)", "bound": "alu",
                    "achieved": ach / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                    "traffic": None, "hbm_frac": byts / t / 1e9 / hbm,
                    "peak_source": "library FP64 FMA probe on this GPU"}
        ach = byts / t
        return {"kernel": "fast_solve (FP32; per application)", "bound": "hbm", "achieved": ach / 1e9,
                "peak": hbm, "unit": "GB/s", "frac": ach / 1e9 / hbm, "traffic": None,
                "alu_frac": flops / t / fp32_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    if phase == "arnoldi":
        # per Arnoldi step: one MGS chain over nrhs vectors
        steps = max(1, phases["givens"]["launches"])
        t = ph["ms"] * 1e-3 / steps
        flops = costs["arnoldi_flops"] * nrhs
        ach = flops / t
        return {"kernel": "arnoldi_mgs (one Arnoldi step)", "bound": "alu", "achieved": ach / 1e12,
                "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": None,
                "hbm_frac": costs["arnoldi_bytes"] * nrhs / t / 1e9 / hbm,
                "peak_source": "library FP64 FMA probe on this GPU"}
    steps = max(1, phases["givens"]["launches"])
    t = ph["ms"] * 1e-3 / steps
    byts = 16.0 * nc * nrhs
    return {"kernel": "schur_matvec", "bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": byts / t / 1e9 / hbm, "traffic": None}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
