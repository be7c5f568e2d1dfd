"""Summaries of Nsight Compute CSV output, small enough to commit as text.

  python -m paper_2509_23180_gb300.ncu_summary launches <launches.csv>
      per kernel: launches, total device time, share, average (from a
      `--metrics gpu__time_duration.sum --csv` launch list)
  python -m paper_2509_23180_gb300.ncu_summary raw <raw.csv>
      per captured launch: duration, DRAM bytes read+write, DRAM throughput,
      FP64/FP32 pipe and issue utilisation, occupancy, registers, stalls and,
      where captured, instruction counts by class (from
      `ncu -i <report> --page raw --csv`)
"""
from __future__ import annotations

import csv
import re
import sys
from collections import defaultdict

UNIT = {"nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0, "ns": 1e-9, "us": 1e-6, "ms": 1e-3,
        "s": 1.0, "B": 1.0,
        "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}


def short(name: str) -> str:
    name = re.sub(r"\(.*", "", name)
    name = name.replace("fpg::<unnamed>::", "").replace("void ", "")
    return name.strip()


def launches(path: str) -> str:
    rows = list(csv.reader(open(path)))
    hdr = None
    agg = defaultdict(lambda: [0, 0.0])
    for r in rows:
        if "Kernel Name" in r:
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        if d.get("Metric Name") != "gpu__time_duration.sum":
            continue
        v = float(d["Metric Value"].replace(",", "")) * UNIT.get(d.get("Metric Unit", "nsecond"), 1e-9)
        k = short(d["Kernel Name"])
        agg[k][0] += 1
        agg[k][1] += v
    tot = sum(v[1] for v in agg.values()) or 1.0
    out = [f"{'kernel':58s} {'launches':>8s} {'total_ms':>10s} {'share':>7s} {'avg_us':>9s}"]
    for k, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        out.append(f"{k[:58]:58s} {c:8d} {t * 1e3:10.3f} {100 * t / tot:6.1f}% {t / c * 1e6:9.2f}")
    out.append(f"{'total':58s} {sum(v[0] for v in agg.values()):8d} {tot * 1e3:10.3f}")
    return "\n".join(out)


WANT = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "dram_read"),
    ("dram__bytes_write.sum", "dram_write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "dram_pct"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "sm_pct"),
    ("sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active", "fp64_pipe_pct"),
    ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active", "fp64_cycles_pct"),
    ("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "fma_cycles_pct"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "occupancy_pct"),
    ("sm__inst_issued.avg.pct_of_peak_sustained_active", "issue_pct"),
    ("launch__registers_per_thread", "regs"),
    ("launch__grid_size", "grid"),
    ("launch__occupancy_limit_registers", "occ_limit_regs"),
    ("launch__occupancy_limit_shared_mem", "occ_limit_smem"),
    ("l1tex__data_pipe_lsu_wavefronts_mem_shared.sum.pct_of_peak_sustained_elapsed", "smem_pct"),
    ("smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio", "stall_barrier"),
    ("smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "stall_long_sb"),
    ("smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", "stall_short_sb"),
    ("smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio", "stall_math"),
    ("smsp__average_warps_issue_stalled_wait_per_issue_active.ratio", "stall_wait"),
    ("smsp__average_warps_issue_stalled_mio_throttle_per_issue_active.ratio", "stall_mio"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue_active_pct"),
]

# instruction counts, printed in millions; the FP32 classes are summed into paired
# (FFMA2, FADD2, FMUL2: two binary32 lanes each) and scalar instructions
COUNTS = [
    ("smsp__inst_executed.sum", "warp_inst"),
    ("smsp__sass_thread_inst_executed.sum", "thread_inst"),
    ("smsp__sass_thread_inst_executed_op_integer_pred_on.sum", "integer"),
    ("smsp__sass_thread_inst_executed_op_memory_pred_on.sum", "memory"),
]
FP32_PAIRED = ["ffma2", "fadd2", "fmul2"]
FP32_SCALAR = ["ffma", "fadd", "fmul"]


def raw(path: str) -> str:
    rows = list(csv.reader(open(path)))
    if len(rows) < 3:
        return "(empty)"
    hdr, units = rows[0], rows[1]
    col = {h: i for i, h in enumerate(hdr)}
    out = []
    for r in rows[2:]:
        if len(r) != len(hdr):
            continue
        name = short(r[col.get("Kernel Name", 0)])
        parts = [name]
        for metric, label in WANT:
            i = col.get(metric)
            if i is None or not r[i]:
                continue
            try:
                v = float(r[i].replace(",", ""))
            except ValueError:
                continue
            u = units[i]
            if metric == "gpu__time_duration.sum":
                v *= UNIT.get(u, 1e-9) * 1e6
                parts.append(f"{label}={v:.2f}us")
            elif metric.startswith("dram__bytes"):
                v *= UNIT.get(u, 1.0)
                parts.append(f"{label}={v / 1e6:.3f}MB")
            else:
                parts.append(f"{label}={v:.2f}")

        def value(metric):
            i = col.get(metric)
            if i is None or not r[i]:
                return None
            try:
                return float(r[i].replace(",", ""))
            except ValueError:
                return None

        for metric, label in COUNTS:
            v = value(metric)
            if v is not None:
                parts.append(f"{label}={v / 1e6:.1f}M")
        for label, ops in (("fp32_paired", FP32_PAIRED), ("fp32_scalar", FP32_SCALAR)):
            vals = [value(f"smsp__sass_thread_inst_executed_op_{o}_pred_on.sum") for o in ops]
            if any(v is not None for v in vals):
                parts.append(f"{label}={sum(v or 0.0 for v in vals) / 1e6:.1f}M")
        out.append("  ".join(parts))
    return "\n".join(out)


def main(argv):
    if len(argv) < 3 or argv[1] not in ("launches", "raw"):
        print(__doc__)
        return 2
    print(launches(argv[2]) if argv[1] == "launches" else raw(argv[2]))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
