"""bench.py's host-side pieces (CPU only): the reference arm's JSON line on a small
workload, the committed DRAM-traffic lookup and its invalidation, the oracle
baseline helper of the widening lines, the algorithmic work behind the roofline,
the choice of the dominant kernel and its peak, and the clock-sample summary."""
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
    nrhs = int(committed["nrhs"])  # right-hand sides of one launch (one domain)
    t = bench.traffic_for("k_arnoldi_cluster_reg", args, nrhs)
    if committed["src"] == bench.source_hash("k_arnoldi_cluster_reg"):
        assert t == float(committed["dram_bytes"])
    else:
        assert t is None
    assert bench.traffic_for("k_arnoldi_cluster_reg", args, nrhs + 1) is None
    assert bench.traffic_for("k_arnoldi_cluster_reg", SimpleNamespace(n=512, precision=64, seeds=10)) is None
    assert bench.traffic_for("k_not_a_kernel", args) is None


def test_cpu_baseline_helper():
    import bench
    import workloads as W
    from oracle import strip
    out = bench.cpu_baseline_of(lambda: strip.assemble(2, 4, 0.0),
                                np.stack([W.strip_fourier_rhs(2, 4, s) for s in range(2)]), "tiny chain")
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == 1 and "tiny chain" in out["sample"]


def test_arnoldi_algorithmic_work_per_point():
    """The roofline's algorithmic work of one Arnoldi step per centre point:
    8(j+1)+16 bytes and 4(j+1)+12 flops at the cycle's mean index j = m/2, i.e.
    144 B and 76 flops for m = 30 (94.4 MB and 49.8 MFLOP per launch of 10
    right-hand sides of 256^2)."""
    import bench
    c = bench.algorithmic_costs(256, 76.6, 30)
    nc = 256 * 256
    assert c["arnoldi_bytes"] == 144.0 * nc and c["arnoldi_flops"] == 76.0 * nc
    assert c["arnoldi_bytes"] * 10 == 94371840.0 and c["arnoldi_flops"] * 10 == 49807360.0
    short = bench.algorithmic_costs(64, 9.0, 30)      # fewer steps than m: j averages over them
    assert short["arnoldi_flops"] == (4.0 * (4.5 + 1) + 12.0) * 64 * 64


def test_roofline_picks_the_dominant_kernel_and_divides_by_its_peak():
    import bench
    args = SimpleNamespace(n=256, precision=64, seeds=10)
    costs = bench.algorithmic_costs(256, 76.6, 30)
    phases = {"arnoldi": {"ms": 17.2, "launches": 180}, "dst_forward": {"ms": 9.8, "launches": 90},
              "thomas": {"ms": 3.6, "launches": 90}, "dst_inverse": {"ms": 10.0, "launches": 90}}
    r = bench.roofline(phases, costs, args, {"hbm_gbs": 6774.0}, 1.05e12, 75e12, 10)
    assert r["phase"] == "arnoldi" and r["kernel"] == "k_arnoldi_cluster_reg" and r["bound"] == "alu"
    t = 17.2e-3 / 180
    assert abs(r["achieved"] - 49807360.0 / t / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1.05) < 1e-12 and r["unit"] == "TFLOP/s"
    # FP32 fast solve dominating: HBM-bound line against the measured copy bandwidth
    args32 = SimpleNamespace(n=256, precision=32, seeds=10)
    phases32 = {"arnoldi": {"ms": 1.0, "launches": 10}, "dst_forward": {"ms": 5.0, "launches": 10}}
    r32 = bench.roofline(phases32, costs, args32, {"hbm_gbs": 6774.0}, 1.05e12, 75e12, 10)
    assert r32["bound"] == "hbm" and r32["unit"] == "GB/s" and r32["peak"] == 6774.0
    assert abs(r32["achieved"] - 12 * 256 * 256 * 10 / 5e-4 / 1e9) < 1e-9


def test_clock_summary_reads_reasons_and_median(tmp_path):
    import bench
    csv = tmp_path / "clocks.csv"
    csv.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                   "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "garbage line\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = object(), str(csv)
    out = s.summary()
    assert out == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}


def test_oracle_pool_splits_the_work_and_matches_the_direct_solve():
    """The CPU leg on several host cores: the workload's right-hand sides split
    over spawn-started workers (each factors K for its share) give exactly the
    oracle's direct solutions, every right-hand side once."""
    import bench
    import workloads as W
    from oracle import direct, operator
    n = 12
    f_by_kappa = {k: W.rhs_batch("cross", n, [0, 1, 2], kind="fourier") for k in (0.0, -10.0)}
    pool = bench.OraclePool(3)
    try:
        tasks = pool.split("cross", n, f_by_kappa)
        assert sum(t[3].shape[0] for t in tasks) == 6 and {t[2] for t in tasks} == {0.0, -10.0}
        dt, sols = pool.run(tasks)
        assert dt > 0
        for (g, nn, kappa, f), P in zip(tasks, sols):
            want = direct.Factor(operator.assemble(g, nn, kappa)).solve(f)
            assert np.allclose(P, want, rtol=1e-13, atol=1e-16)
        out = bench.cpu_baseline(SimpleNamespace(n=n), f_by_kappa, pool)
        assert out["kind"] == "oracle" and out["value"] > 0 and 1 <= out["cores"] <= 3
    finally:
        pool.close()


def test_error_stats_sees_one_wrong_block():
    """The bench's error statement is element-wise: a mistake confined to one arm
    shows at its own size in max-abs and in the worst block."""
    import bench
    import workloads as W
    n = 10
    R = W.rhs_batch("cross", n, [4], kind="fourier")[0]
    P = R.copy()
    off = n * n  # W arm follows the centre
    P[off + 3] += 1e-6 * np.abs(R).max()
    e = bench.error_stats(P, R, "cross", n)
    assert e["worst_block"]["block"] == "W"
    assert abs(e["maxabs_rel"] - 1e-6) < 1e-9 and e["rel_2norm"] < e["maxabs_rel"]


def test_parity_helper_is_element_wise():
    """The GPU tests' error measure sees a mistake on one interface line that the
    2-norm of the whole vector dilutes, and judges near-zero parts at 1% of the
    solution's scale."""
    from tests import parity
    import workloads as W
    n = 16
    R = W.rhs_batch("cross", n, [2], kind="fourier")[0]
    P = R.copy()
    line = dict(parity.part_slices("cross", n))["W|C"]
    P[line] += 1e-8 * np.abs(R).max()
    assert parity.rel(P, R) >= 0.99e-8 and parity.norm_rel(P, R) < 0.5 * parity.rel(P, R)
    errs = parity.part_errors(P, R, "cross", n)
    assert errs["W|C"] > 1e-9 and errs["C"] == 0.0 and errs["E|C"] == 0.0
    # a part of near-zero values: its error is measured against 1% of max|R|
    Z = R.copy()
    Z[line] = 1e-14
    Pz = Z.copy()
    Pz[line] += 1e-12 * np.abs(Z).max()
    assert parity.part_errors(Pz, Z, "cross", n)["W|C"] <= 1e-10
