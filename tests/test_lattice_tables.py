"""The library's host tables of the general concatenated geometry (CPU only;
needs nvcc): a small host program built from the library's own fpg_lattice_host.h
prints the layout and the neighbour / coupling tables, and each is checked
against the oracle (oracle/lattice.py) built independently from the squares:
  * block counts and offsets equal the oracle's block listing;
  * the global neighbour table gnbr is exactly the off-diagonal pattern of the
    oracle's K (every neighbour pair, in both directions, nothing else);
  * the coupled set's table nbr is that pattern restricted to the coupled set,
    anb the coupled set's neighbours among the independent squares, gcn the
    reverse link, so that (nbr, anb) and gcn are R_cc, R_ca and R_ac of K;
  * each face lists the coupled boundary line that touches its independent
    square, in the order of the independent square's own line.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import lattice as LT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_23180_gb300", "csrc")
CASES = [("square2x2", 4), ("L5", 3), ("T6", 5), ("cross", 4), ("domino", 3),
         ("ring8", 3), ("plus3x3", 2)]
MASKS = dict(W.LATTICE_EXAMPLES)
MASKS["ring8"] = sum(1 << (i + 8 * j) for i in range(3) for j in range(3) if (i, j) != (1, 1))
MASKS["plus3x3"] = sum(1 << (i + 8 * j) for i in range(3) for j in range(3))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "fpg_lattice_host.h"
using namespace fpg;
int main(int argc, char** argv) {
  const unsigned long long mask = strtoull(argv[1], nullptr, 10);
  const int n = atoi(argv[2]);
  LatticeGeom g;
  if (!lattice_shape(mask, n, &g)) { printf("BAD\n"); return 0; }
  printf("SHAPE %d %d %d %d %d %d %lld %lld %lld %lld\n", g.ncsq, g.nlinks, g.njunc, g.nfaces, g.nwe, g.nsn,
         g.nc, g.ntot, g.link_base, g.junc_base);
  printf("SQ");
  for (int k = 0; k < g.ncsq; ++k) printf(" %lld", g.sq_off[k]);
  printf("\nWE");
  for (int k = 0; k < g.nwe; ++k) printf(" %lld", g.we_off[k]);
  printf("\nSN");
  for (int k = 0; k < g.nsn; ++k) printf(" %lld", g.sn_off[k]);
  printf("\n");
  LatticeHost t;
  lattice_tables(mask, n, (n + 1.0) * (n + 1.0), -2.0, &t);
  for (size_t i = 0; i < t.gnbr.size(); ++i)
    printf("G %d %d %d %d %d\n", t.gnbr[i].x, t.gnbr[i].y, t.gnbr[i].z, t.gnbr[i].w, t.gcn[i]);
  for (size_t i = 0; i < t.nbr.size(); ++i)
    printf("C %d %d %d %d %d %d %d %d\n", t.nbr[i].x, t.nbr[i].y, t.nbr[i].z, t.nbr[i].w, t.cf[i].x, t.cf[i].y,
           t.anb[i].x, t.anb[i].y);
  for (size_t f = 0; f < t.faces.size(); ++f) printf("F %d %d\n", t.faces[f].x, t.faces[f].y);
  for (size_t s = 0; s < t.lpiv.size(); ++s) printf("L %a\n", t.lpiv[s]);
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("lattice")
    (d / "main.cu").write_text(PROGRAM)
    out = d / "lat"
    flags = ["-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
             "-gencode", "arch=compute_103a,code=sm_103a"]
    subprocess.run([nvcc, *flags, str(d / "main.cu"), "-o", str(out)], check=True, capture_output=True, timeout=600)
    return str(out)


def run(exe, mask, n):
    txt = subprocess.run([exe, str(mask), str(n)], check=True, capture_output=True, text=True, timeout=60).stdout
    rec = {"G": [], "C": [], "F": [], "L": []}
    for line in txt.splitlines():
        tag, *vals = line.split()
        if tag in rec:
            rec[tag].append([float.fromhex(v) for v in vals] if tag == "L" else list(map(int, vals)))
        else:
            rec[tag] = list(map(int, vals))
    return rec


@pytest.mark.parametrize("name,n", CASES)
def test_tables_match_the_oracle(exe, name, n):
    mask = MASKS[name]
    rec = run(exe, mask, n)
    br = LT.block_ranges(mask, n)
    coupled, indep = LT.classify(mask)
    nc = LT.coupled_size(mask, n)
    ncsq, nlinks, njunc, nfaces, nwe, nsn, nc_l, ntot, link_base, junc_base = rec["SHAPE"]
    assert (ncsq, nlinks, njunc, nfaces) == (len(coupled), len(LT.links(mask)), len(LT.junctions(mask)), len(indep))
    assert nc_l == nc and ntot == sum(b[6] for b in br)
    assert link_base == len(coupled) * n * n and junc_base == link_base + nlinks * n
    assert rec["SQ"] == [b[5] for b in br if b[0][0] == "Q"]
    arms = [b for b in br if b[0][0] == "A"]
    we = [b[5] for b in arms if b[3] == n + 1]
    sn = [b[5] for b in arms if b[3] == n]
    assert (nwe, nsn) == (len(we), len(sn)) and rec["WE"] == we and rec["SN"] == sn
    # gnbr: the off-diagonal pattern of K, neighbour by neighbour
    K = LT.assemble(mask, n, -2.0).tocsr()
    pts = LT.block_order_points(mask, n)
    index = {p: k for k, p in enumerate(pts)}
    G = np.array(rec["G"])
    for g, (I, J) in enumerate(pts):
        want = [index.get(q, -1) for q in ((I - 1, J), (I + 1, J), (I, J - 1), (I, J + 1))]
        assert list(G[g, :4]) == want, (g, I, J)
        cols = set(K.indices[K.indptr[g]:K.indptr[g + 1]]) - {g}
        assert cols == {q for q in want if q >= 0}
        # gcn: an independent square's point next to the coupled set
        cn = [q for q in want if 0 <= q < nc]
        assert G[g, 4] == (cn[0] if g >= nc and cn else -1)
    C = np.array(rec["C"])
    for i in range(nc):
        nb = list(G[i, :4])
        assert list(C[i, :4]) == [q if 0 <= q < nc else -1 for q in nb]
        assert sorted(q for q in C[i, 6:8] if q >= 0) == sorted(q for q in nb if q >= nc)
    # faces: the coupled line touching each independent square, position by position
    F = rec["F"]
    assert len(F) == len(indep)
    for f, ((sq, d), (off, side)) in enumerate(zip(indep.items(), F)):
        hits = [(i, c) for i in range(nc) for c in C[i, 4:6] if c >= 0 and c // n == f]
        assert len(hits) == n and sorted(c % n for _, c in hits) == list(range(n))
        for i, c in hits:
            arm_pts = [q for q in C[i, 6:8] if q >= 0]
            assert len(arm_pts) >= 1  # a coupled line point touches the independent square's line
    # the links' pivots solve tridiag(delta, -4 delta + kappa, delta)
    delta = (n + 1.0) ** 2
    r = np.array(rec["L"])[:, 0]
    T = np.diag(np.full(n, -4 * delta - 2.0)) + np.diag(np.full(n - 1, delta), 1) + np.diag(np.full(n - 1, delta), -1)
    b = np.arange(1.0, n + 1)
    y = np.zeros(n)
    for s in range(n):
        y[s] = r[s] * (b[s] - delta * (y[s - 1] if s else 0.0))
    x = np.zeros(n)
    for s in range(n - 1, -1, -1):
        x[s] = y[s] - delta * r[s] * (x[s + 1] if s < n - 1 else 0.0)
    assert np.allclose(T @ x, b, rtol=1e-12, atol=1e-12)


def test_disconnected_mask_is_refused(exe):
    txt = subprocess.run([exe, str((1 << 0) | (1 << 2)), "4"], check=True, capture_output=True, text=True).stdout
    assert txt.strip() == "BAD"
