"""bench.py's host-side pieces (CPU only): the reference arm's JSON line on a small
workload, the committed DRAM-traffic lookup and its invalidation, and the oracle
baseline helper of the widening lines."""
import json
import os
import subprocess
import sys
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                          "--seeds", "2", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "dtype", "data", "config"):
        assert key in line, key


def test_traffic_lookup_follows_sources_and_workload():
    """The committed capture is used only while the kernel's sources hash as when it
    was taken, and only for its own workload."""
    import bench
    args = SimpleNamespace(n=256, precision=64, seeds=10)
    committed = None
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        if line.startswith("kernel=k_arnoldi_cluster_reg "):
            committed = dict(kv.split("=", 1) for kv in line.split())
    assert committed is not None
    t = bench.traffic_for("k_arnoldi_cluster_reg", args)
    if committed["src"] == bench.source_hash("k_arnoldi_cluster_reg"):
        assert t == float(committed["dram_bytes"])
    else:
        assert t is None
    assert bench.traffic_for("k_arnoldi_cluster_reg", SimpleNamespace(n=512, precision=64, seeds=10)) is None
    assert bench.traffic_for("k_not_a_kernel", args) is None


def test_cpu_baseline_helper():
    import bench
    import workloads as W
    from oracle import strip
    out = bench.cpu_baseline_of(lambda: strip.assemble(2, 4, 0.0),
                                np.stack([W.strip_fourier_rhs(2, 4, s) for s in range(2)]), "tiny chain")
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == 1 and "tiny chain" in out["sample"]
