"""The compile-time twiddles of the register DFTs (CPU only; needs nvcc).

dl::turn_sincos(m, R) gives sin and cos of 2 pi m / R: the fraction m / R is
reduced exactly to one octant and a 14-term Taylor series is summed in double.
Every radix-R register DFT and every size-specialised DST kernel folds these
values in as constants.  The test compiles the library's own header for the
host, evaluates the function for every m of a set of lengths (and a few values
at compile time, which is how the kernels use it, to show both agree), and
compares against 40-digit values: the error stays within 3 ulp of the exact
value (measured worst 2.71 ulp, 2.9e-16 absolute), and the exact zeros and
ones of the circle (m R / 4 multiples) come out exact.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_23180_gb300", "csrc")
LENGTHS = [2, 3, 4, 5, 7, 8, 13, 16, 19, 25, 27, 41, 43, 64, 256, 257, 512, 513, 1024, 1025, 2048]
CONSTEXPR = [(1, 257), (17, 257), (100, 513), (3, 16), (5, 13), (-7, 25), (611, 1025), (40, 43)]

PROGRAM = r"""
#include <cstdio>
#include "fpg_dstline.cuh"
int main() {
  const long long Rs[] = {%(lengths)s};
  for (long long R : Rs)
    for (long long m = -R; m < 2 * R; ++m)
      std::printf("%%lld %%lld %%a %%a\n", m, R, fpg::dl::turn_sincos(m, R, true),
                  fpg::dl::turn_sincos(m, R, false));
%(constexpr)s
  return 0;
}
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("twiddles")
    ce = "\n".join(
        f"  {{ constexpr double s = fpg::dl::turn_sincos({m}, {R}, true), c = fpg::dl::turn_sincos({m}, {R}, false);\n"
        f"    std::printf(\"C %lld %lld %a %a\\n\", {m}LL, {R}LL, s, c); }}" for m, R in CONSTEXPR)
    src = d / "tw.cu"
    src.write_text(PROGRAM % {"lengths": ", ".join(map(str, LENGTHS)), "constexpr": ce})
    exe = d / "tw"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-gencode", "arch=compute_103a,code=sm_103a", str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    run, comp = {}, {}
    for line in out.splitlines():
        parts = line.split()
        dst = comp if parts[0] == "C" else run
        if parts[0] == "C":
            parts = parts[1:]
        dst[(int(parts[0]), int(parts[1]))] = (float.fromhex(parts[2]), float.fromhex(parts[3]))
    return run, comp


def test_compile_time_values_equal_host_values(table):
    run, comp = table
    assert len(comp) == len(CONSTEXPR)
    for key, v in comp.items():
        assert run[key] == v, key


def test_twiddles_within_three_ulp(table):
    run, _ = table
    mpmath.mp.dps = 40
    worst = 0.0
    for (m, R), (s, c) in run.items():
        a = 2 * mpmath.pi * m / R
        for got, ex in ((s, mpmath.sin(a)), (c, mpmath.cos(a))):
            if (4 * m) % R == 0:                      # 0, +-1 on the axes: exact
                assert got == float(mpmath.nint(ex)), (m, R)
                continue
            ulp = np.spacing(abs(float(ex)))
            err = float(abs(mpmath.mpf(got) - ex)) / ulp
            worst = max(worst, err)
            assert err <= 3.0, (m, R, got, err)
    assert worst > 0.5  # the sum is not correctly rounded; the bound above is what holds


def test_periodicity_and_symmetry_are_exact(table):
    run, _ = table
    for (m, R), (s, c) in run.items():
        if 0 <= m < R:
            assert run[(m - R, R)] == (s, c) and run[(m + R, R)] == (s, c)
            assert run[(-m, R)] == (-s, c)  # (a signed zero compares equal to zero)
