"""The batch runtime's pool allocator (`PoolFreeList`, csrc/fpg_pool.h), the native code
that carves resident domains out of the caller's one device pool (CPU only; needs g++).

A host program drives the allocator through random sequences of requests and returns
and checks every step against an independent model of the pool: one flag per 256-byte
unit.  Checked after each operation: the free ranges are sorted, disjoint, never
adjacent (coalesced), inside the pool and 256-byte aligned; they cover exactly the units
the model has free; a granted range is first fit (no free range before it could hold the
request) and lies on free units only; a refusal happens only when no free range holds
the request.  When everything has been returned the pool is one range again.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_23180_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <random>
#include <vector>
#include "fpg_pool.h"

static int fail(const char* what, int step) { std::printf("FAIL %s at step %d\n", what, step); return 1; }

int main() {
  long long granted = 0, refused = 0;
  for (int trial = 0; trial < 40; ++trial) {
    std::mt19937_64 rng(1234 + trial);
    const size_t units = 64 + rng() % 512, pool = units * 256;
    fpg::PoolFreeList fl;
    fl.reset(pool);
    std::vector<char> used(units, 0);
    std::vector<std::pair<size_t, size_t>> live;  // (offset, bytes as requested)
    for (int step = 0; step < 3000; ++step) {
      const bool give = !live.empty() && (rng() % 100) < 45;
      if (give) {
        const size_t k = rng() % live.size();
        const auto a = live[k];
        live.erase(live.begin() + k);
        fl.give(a.first, a.second);
        for (size_t u = a.first / 256; u < (a.first + fpg::align256(a.second)) / 256; ++u) used[u] = 0;
      } else {
        const size_t bytes = 1 + rng() % (48 * 256);  // not a multiple of 256 in general
        const size_t need = fpg::align256(bytes);
        // the model's first fit: the lowest free range of the allocator that holds `need`
        size_t expect = (size_t)-1;
        for (const auto& r : fl.ranges)
          if (r.second >= need) { expect = r.first; break; }
        size_t off = 0;
        if (fl.take(bytes, &off)) {
          if (off != expect) return fail("not first fit", step);
          if (off % 256 || off + need > pool) return fail("range outside the pool or unaligned", step);
          for (size_t u = off / 256; u < (off + need) / 256; ++u) {
            if (used[u]) return fail("granted a used unit", step);
            used[u] = 1;
          }
          live.push_back({off, bytes});
          ++granted;
        } else {
          if (expect != (size_t)-1) return fail("refused although a range fits", step);
          ++refused;
        }
      }
      // invariants of the free list against the model
      std::vector<char> fr(units, 0);
      size_t prev_end = 0;
      for (size_t i = 0; i < fl.ranges.size(); ++i) {
        const auto r = fl.ranges[i];
        if (r.second == 0 || r.first % 256 || r.second % 256) return fail("empty or unaligned range", step);
        if (r.first + r.second > pool) return fail("range past the pool", step);
        if (i > 0 && r.first <= prev_end) return fail("ranges unsorted, overlapping or not coalesced", step);
        prev_end = r.first + r.second;
        for (size_t u = r.first / 256; u < prev_end / 256; ++u) fr[u] = 1;
      }
      for (size_t u = 0; u < units; ++u)
        if (fr[u] == used[u]) return fail("free list and model disagree", step);
    }
    for (const auto& a : live) fl.give(a.first, a.second);
    if (fl.ranges.size() != 1 || fl.ranges[0].first != 0 || fl.ranges[0].second != pool)
      return fail("pool not whole after every range came back", -1);
  }
  std::printf("OK %lld %lld\n", granted, refused);
  return 0;
}
"""


def test_pool_allocator_against_a_unit_model(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    src = tmp_path / "pool.cpp"
    exe = tmp_path / "pool"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-std=c++17", "-O2", f"-I{CSRC}", str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120).stdout.split()
    assert out[0] == "OK", " ".join(out)
    granted, refused = int(out[1]), int(out[2])
    assert granted > 10000 and refused > 1000  # both paths ran many times
