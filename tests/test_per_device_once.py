"""The library's once-per-device host set-up (`PerDeviceOnce`, csrc/fpg_once.h) under
several host threads (CPU only; needs g++ and the CUDA headers).

A kernel that needs more than 48 KB of dynamic shared memory must have its limit raised
on a device before its first launch there.  The library raises it in a block guarded by
`PerDeviceOnce`, and host threads (the concurrent bench, the end-to-end pass's thread
pool, a caller's own threads) may reach that block together.  The test compiles the
header into a host program with a stand-in `cudaGetDevice` and runs 16 threads through
the guarded block; the block sleeps, so a thread that passed it early would see its work
unfinished.  Checked: the block runs exactly once per device; every thread, once past
the `if`, sees the block's work complete; a device ordinal beyond the per-device record
(64 and up) runs the block on every call.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_23180_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <chrono>
#include <cstdio>
#include <thread>
#include <vector>
#include "fpg_once.h"

static std::atomic<int> g_device{0};
extern "C" cudaError_t cudaGetDevice(int* device) {  // stand-in for the runtime's
  *device = g_device.load();
  return cudaSuccess;
}

int main() {
  for (int dev : {0, 3, 70}) {
    g_device.store(dev);
    fpg::PerDeviceOnce once_per_device;
    std::atomic<int> runs{0}, early{0};
    std::atomic<bool> ready{false};
    std::vector<std::thread> th;
    for (int t = 0; t < 16; ++t)
      th.emplace_back([&] {
        if (auto once = once_per_device.first()) {
          std::this_thread::sleep_for(std::chrono::milliseconds(30));
          ready.store(true);
          runs.fetch_add(1);
        }
        if (!ready.load()) early.fetch_add(1);
      });
    for (auto& x : th) x.join();
    // a later call on the same device does not run the block again (below 64)
    bool again = false;
    if (auto once = once_per_device.first()) again = true;
    std::printf("DEV %d RUNS %d EARLY %d AGAIN %d\n", dev, runs.load(), early.load(), again ? 1 : 0);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime_api.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("once")
    src = d / "once.cpp"
    exe = d / "once"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", f"-I{CSRC}", f"-I{CUDA_INC}", str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    rows = {}
    for line in out.splitlines():
        f = line.split()
        rows[int(f[1])] = dict(runs=int(f[3]), early=int(f[5]), again=int(f[7]))
    return rows


@pytest.mark.parametrize("dev", [0, 3])
def test_block_runs_once_and_no_thread_passes_before_it_ends(report, dev):
    r = report[dev]
    assert r["runs"] == 1
    assert r["early"] == 0
    assert r["again"] == 0


def test_device_past_the_record_runs_the_block_every_time(report):
    r = report[70]
    assert r["runs"] == 16 and r["again"] == 1
