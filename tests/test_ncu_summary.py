"""The ncu CSV summaries behind the committed profiles (CPU only): the launch
list's per-kernel launches, total time, share and average with ncu's unit
strings, and the raw-page per-launch line."""
from paper_2509_23180_gb300 import ncu_summary as S

LAUNCH_HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
              '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(i, kernel, unit, value):
    return (f'"{i}","1","python3","127.0.0.1","{kernel}","1","13","(256, 1, 1)","(160, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","gpu__time_duration.sum","{unit}","{value}"\n')


def test_launch_list_aggregates_per_kernel(tmp_path):
    p = tmp_path / "launches.csv"
    p.write_text("==PROF== Connected to process 1\n" + LAUNCH_HDR
                 + _row(0, "void fpg::<unnamed>::k_arnoldi_cluster_reg<16>(const double *, int)", "usecond", "90")
                 + _row(1, "void fpg::<unnamed>::k_arnoldi_cluster_reg<16>(const double *, int)", "usecond", "110")
                 + _row(2, "void dl::k_dst_lines_fwd<double, 257>(const double *)", "nsecond", "50,000")
                 + _row(3, "k_givens(double *)", "msecond", "0.05")
                 + '"4","1","python3"\n')                     # a truncated row is skipped
    lines = S.launches(str(p)).splitlines()
    rows = {l.split()[0]: l.split() for l in lines[1:]}
    arn = rows["k_arnoldi_cluster_reg<16>"]
    assert arn[1] == "2" and float(arn[2]) == 0.2 and arn[3] == "66.7%" and float(arn[4]) == 100.0
    dst = rows["dl::k_dst_lines_fwd<double,"]
    assert dst[-4] == "1" and float(dst[-3]) == 0.05 and dst[-2] == "16.7%"
    assert rows["k_givens"][1] == "1" and float(rows["k_givens"][2]) == 0.05
    total = rows["total"]
    assert total[1] == "4" and float(total[2]) == 0.3
    assert lines[1].startswith("k_arnoldi_cluster_reg")      # sorted by total time


def test_raw_page_line(tmp_path):
    p = tmp_path / "raw.csv"
    p.write_text('"Kernel Name","gpu__time_duration.sum","dram__bytes_read.sum","dram__bytes_write.sum",'
                 '"launch__registers_per_thread"\n'
                 '"","usecond","Mbyte","Kbyte","register/thread"\n'
                 '"void fpg::<unnamed>::k_thomas_reg<double, 9>(double *)","48.5","12.5","500","64"\n')
    out = S.raw(str(p))
    assert out == "k_thomas_reg<double, 9>  duration=48.50us  dram_read=12.500MB  dram_write=0.500MB  regs=64.00"


def test_usage_without_arguments():
    assert S.main(["ncu_summary"]) == 2


def test_raw_page_instruction_mix(tmp_path):
    p = tmp_path / "raw.csv"
    cols = ["smsp__inst_executed.sum", "smsp__sass_thread_inst_executed_op_integer_pred_on.sum",
            "smsp__sass_thread_inst_executed_op_ffma2_pred_on.sum", "smsp__sass_thread_inst_executed_op_fadd2_pred_on.sum",
            "smsp__sass_thread_inst_executed_op_ffma_pred_on.sum"]
    p.write_text('"Kernel Name",' + ",".join(f'"{c}"' for c in cols) + "\n"
                 + '"",' + ",".join('"inst"' for _ in cols) + "\n"
                 + '"k_x(float *)","28,880,000","343,000,000","200,000,000","20,000,000","5,000,000"\n')
    out = S.raw(str(p))
    assert out == "k_x  warp_inst=28.9M  integer=343.0M  fp32_paired=220.0M  fp32_scalar=5.0M"
