"""The library's host-side tables (CPU only; needs nvcc): the DST-I plan of a
line length, Rader's permutations and kernel, the sine table, and the Thomas
pivots of every mode.  A small host program built from the library's own header
(fpg_host_tables.h) prints them, and each is checked by an independent route:
  * the plan's radices multiply to its FFT length, the mode follows from p = n + 1
    (Stockham when p factors into 4, 2 and odd primes to 43, Rader for such a p - 1
    with p prime, the dense DST otherwise);
  * Rader: pin[b] = g^b mod p with g of order p - 1 (so pin is a permutation of
    1..p-1), pout = its inverse powers, and Bhat = DFT(B)/N (numpy FFT), which
    makes the Rader convolution reproduce numpy's DFT of length p;
  * sinp[j] = sin(pi j / p) within 4 units in the last place of 40-digit values
    (a relative bound, which the folding to the first octant gives), sinp[0] = 0;
  * a Thomas sweep with the printed reciprocal pivots solves tridiag(delta,
    d_k, delta) x = f as LAPACK's banded solver does (scipy), with
    d_k = -4 delta + 2 delta cos(k pi/(n+1)) + kappa (Sec. 2.1, Eq. "trans_subeq");
  * the Neumann (DCT-II) and periodic (real DFT) lines' pivots solve their mode
    systems as LAPACK's banded solver does, with the eigenvalues mu_k taken from
    the oracle's pinned line operators and a Neumann-sided arm's end-row term;
  * the interface table of the reduced Schur form: G(i, j) = T(|i-j|) - H(i+j), built
    from the arm's eigenvalues, equals every arm's R_ca A_a^{-1} R_ac on the centre's
    facing line with A_a^{-1} a sparse LU of the oracle's arm block (a dropped or
    shifted Hankel part is off by about a third).
Rader's tables and the pivots are printed from the heap-free forms
(`rader_tables`, `fill_pivots_into`) that the no-allocation fast solve calls,
and checked identical to what the domain API's `build_plan` / `fill_pivots` give.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_23180_gb300", "csrc")
SIZES = [2, 7, 16, 33, 64, 88, 93, 100, 256, 512, 1024]
PIVOTS = [(8, 5, 81.0, 0.0), (64, 64, 4225.0, -10.0), (256, 257, 66049.0, -3.0)]

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "fpg_host_tables.h"
using namespace fpg;
int main() {
  const int sizes[] = {%(sizes)s};
  for (int n : sizes) {
    HostPlan P = build_plan(n);
    std::printf("PLAN %%d %%d %%d %%d", n, P.mode, P.N, P.nrad);
    for (int i = 0; i < P.nrad; ++i) std::printf(" %%d", P.rad[i]);
    std::printf("\nSINP %%d", n);
    for (double v : P.sinp) std::printf(" %%a", v);
    std::printf("\n");
    if (P.mode == DST_RADER) {
      // the heap-free form the no-allocation entry point calls, into fixed arrays
      static int pin[4096], pout[4096];
      static double bhat[8192];
      rader_tables(n + 1, pin, pout, bhat);
      std::printf("PIN %%d", n);
      for (int b = 0; b < P.N; ++b) std::printf(" %%d", pin[b]);
      std::printf("\nPOUT %%d", n);
      for (int b = 0; b < P.N; ++b) std::printf(" %%d", pout[b]);
      std::printf("\nBHAT %%d", n);
      for (int b = 0; b < 2 * P.N; ++b) std::printf(" %%a", bhat[b]);
      std::printf("\nSAME %%d %%d\n", n, (int)(std::vector<int>(pin, pin + P.N) == P.pin &&
                                              std::vector<int>(pout, pout + P.N) == P.pout &&
                                              std::vector<double>(bhat, bhat + 2 * P.N) == P.Bhat));
    }
  }
  struct Pv { int n, ns; double delta, kappa; };
  const Pv pv[] = {%(pivots)s};
  for (const Pv& q : pv) {
    std::vector<double> r((size_t)q.n * q.ns), rv;
    fill_pivots_into(q.n, q.ns, q.delta, q.kappa, r.data());  // heap-free form (caller storage)
    fill_pivots(q.n, q.ns, q.delta, q.kappa, rv);
    std::printf("SAME %%d %%d\n", q.n, (int)(r == rv));
    std::printf("PIV %%d %%d", q.n, q.ns);
    for (double v : r) std::printf(" %%a", v);
    std::printf("\n");
  }
  // the reduced Schur term of a Dirichlet arm on the centre's facing line:
  // G(i, j) = T(|i - j|) - H(i + j) from the interface table, as the domain stores it
  struct Ct { int n; double kappa; };
  const Ct cts[] = {%(ctabs)s};
  int idx = 0;
  for (const Ct& q : cts) {
    const double delta = (double)(q.n + 1) * (double)(q.n + 1);
    std::vector<double> pa, ct;
    fill_pivots(q.n, q.n + 1, delta, q.kappa, pa);
    fill_ctab(q.n, delta, pa, ct);
    std::printf("CTAB %%d %%d %%a", idx++, q.n, q.kappa);
    for (int i = 0; i < q.n; ++i)
      for (int j = 0; j < q.n; ++j) std::printf(" %%a", ct[i > j ? i - j : j - i] - ct[2 * q.n + 2 + i + j]);
    std::printf("\n");
  }
  // the same for arms with Neumann sides (cell-centred, DCT-II lines, the far end a
  // Dirichlet face half a cell beyond the arm's row 0): H(m) = -T(m + 1)
  idx = 0;
  for (const Ct& q : cts) {
    const double delta = (double)q.n * (double)q.n;
    std::vector<double> pa, ma, ct;
    dct_pivots(q.n, q.n, delta, q.kappa, -delta, 0, pa, ma);
    fill_ctab_dct(q.n, delta, pa, ct);
    std::printf("CTABN %%d %%d %%a", idx++, q.n, q.kappa);
    for (int i = 0; i < q.n; ++i)
      for (int j = 0; j < q.n; ++j) std::printf(" %%a", ct[i > j ? i - j : j - i] - ct[2 * q.n + 2 + i + j]);
    std::printf("\n");
  }
  // Thomas pivots of the Neumann (DCT-II) and periodic (real DFT) lines
  struct Dp { int nt, ns; double delta, kappa, extra; int end; };
  const Dp dps[] = {%(dpivots)s};
  idx = 0;
  for (const Dp& q : dps) {
    std::vector<double> r, m;
    dct_pivots(q.nt, q.ns, q.delta, q.kappa, q.extra, q.end, r, m);
    std::printf("DPIV %%d", idx++);
    for (double v : r) std::printf(" %%a", v);
    for (double v : m) std::printf(" %%a", v);
    std::printf("\n");
  }
  for (int nt : {8, 12, 256}) {
    std::vector<double> W, post;
    dct_tables(nt, W, post);
    std::printf("DCTW %%d", nt);
    for (double v : W) std::printf(" %%a", v);
    for (double v : post) std::printf(" %%a", v);
    std::printf("\n");
  }
  const Pv rps[] = {%(rpivots)s};
  idx = 0;
  for (const Pv& q : rps) {
    std::vector<double> r, m;
    rdft_pivots(q.n, q.ns, q.delta, q.kappa, r, m);
    std::printf("RPIV %%d", idx++);
    for (double v : r) std::printf(" %%a", v);
    for (double v : m) std::printf(" %%a", v);
    std::printf("\n");
  }
  // the one-pass FP32 cluster kernel's tables: sigma_k and the scaled pivot w at the first
  // row of every CTA, with the reciprocal Thomas pivots of the same block beside them
  idx = 0;
  for (int n : {64, 512}) {
    for (double kappa : {0.0, -10.0}) {
      const double delta = (double)(n + 1) * (double)(n + 1);
      std::vector<float> sigma, wseed;
      std::vector<double> r;
      const bool ok = fast_solve_cluster_tables(n, delta, kappa, sigma, wseed);
      fill_pivots(n, n, delta, kappa, r);
      std::printf("CLUS %%d %%d %%a %%d %%d", idx++, n, kappa, (int)ok, kClusterRows);
      for (float v : sigma) std::printf(" %%a", (double)v);
      for (float v : wseed) std::printf(" %%a", (double)v);
      for (double v : r) std::printf(" %%a", v);
      std::printf("\n");
    }
  }
  {
    std::vector<float> sigma, wseed;
    std::printf("CLUSNO 0 %%d %%d\n", (int)fast_solve_cluster_tables(256, 257.0 * 257.0, 0.0, sigma, wseed),
                (int)fast_solve_cluster_tables(1024, 1025.0 * 1025.0, 0.0, sigma, wseed));
  }
  return 0;
}
"""
CTABS = [(4, 0.0), (8, -10.0), (13, -3.0), (16, 0.0)]
# (nt, ns, delta, kappa, extra on an end row, which end): the Neumann rectangle plan
# (no extra) and the Neumann-sided arms (-delta at row 0 or at row ns - 1)
DPIVOTS = [(8, 5, 81.0, 0.0, 0.0, 0), (16, 16, 256.0, -10.0, -256.0, 0), (12, 7, 144.0, -3.0, -144.0, 1)]
# (nt, ns, delta, kappa): periodic lines
RPIVOTS = [(8, 6, 81.0, 0.0), (10, 10, 100.0, -10.0)]

@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("tables")
    pv = ", ".join(f"{{{n}, {ns}, {delta!r}, {kappa!r}}}" for n, ns, delta, kappa in PIVOTS)
    src = d / "tables.cu"
    cts = ", ".join(f"{{{n}, {kappa!r}}}" for n, kappa in CTABS)
    dps = ", ".join(f"{{{a}, {b}, {c!r}, {d!r}, {e!r}, {g}}}" for a, b, c, d, e, g in DPIVOTS)
    rps = ", ".join(f"{{{a}, {b}, {c!r}, {d!r}}}" for a, b, c, d in RPIVOTS)
    src.write_text(PROGRAM % {"sizes": ", ".join(map(str, SIZES)), "pivots": pv, "ctabs": cts,
                              "dpivots": dps, "rpivots": rps})
    probe = d / "modes.cu"
    probe.write_text('#include <cstdio>\n#include "fpg_dst.cuh"\n'
                     'int main() { std::printf("%d %d %d\\n", fpg::DST_DENSE, fpg::DST_STOCKHAM, fpg::DST_RADER); }\n')
    flags = ["-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
             "-gencode", "arch=compute_103a,code=sm_103a"]
    out = {}
    for name in ("tables", "modes"):
        exe = d / name
        subprocess.run([nvcc, *flags, str(d / f"{name}.cu"), "-o", str(exe)], check=True, capture_output=True,
                       timeout=300)
        out[name] = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    modes = dict(zip(("dense", "stockham", "rader"), map(int, out["modes"].split())))
    rec = {}
    for line in out["tables"].splitlines():
        tag, key, *vals = line.split()
        if tag == "SAME":
            rec.setdefault(("SAME", 0), []).append((int(key), int(vals[0])))
            continue
        rec[(tag, int(key))] = vals
    return modes, rec


def test_heap_free_forms_equal_the_vector_forms(tables):
    _, rec = tables
    same = rec[("SAME", 0)]
    assert len(same) == sum(1 for n in SIZES if rec.get(("PIN", n))) + len(PIVOTS)
    assert all(ok == 1 for _, ok in same), same


def _hex(vals):
    return np.array([float.fromhex(v) for v in vals])


def _factors_ok(p):
    m = p
    while m % 2 == 0:
        m //= 2
    for q in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43):
        while m % q == 0:
            m //= q
    return m == 1


def _is_prime(p):
    return p > 1 and all(p % d for d in range(2, int(p ** 0.5) + 1))


@pytest.mark.parametrize("n", SIZES)
def test_plan_mode_and_radices(tables, n):
    modes, rec = tables
    mode, N, nrad, *rad = map(int, rec[("PLAN", n)])
    p = n + 1
    if p > 1 and _factors_ok(p):
        assert mode == modes["stockham"] and N == p
    elif _is_prime(p) and _factors_ok(p - 1):
        assert mode == modes["rader"] and N == p - 1
    else:
        assert mode == modes["dense"] and nrad == 0
        return
    assert len(rad) == nrad and int(np.prod(rad)) == N
    assert all(r in (2, 3, 4, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43) for r in rad)


@pytest.mark.parametrize("n", SIZES)
def test_sine_table(tables, n):
    _, rec = tables
    p = n + 1
    s = _hex(rec[("SINP", n)])
    assert len(s) == p
    mpmath.mp.dps = 40
    assert s[0] == 0.0
    # relative accuracy: the folding to the first octant is exact in integers, so each
    # entry is the sine or cosine of an angle in [0, pi/4] whose only error is the
    # rounding of pi q/den (a few units in its last place), which the sine passes on
    # relatively and the cosine damps; measured worst 2.37 * 2^-53 over these sizes,
    # and the bound of 4 * 2^-53 leaves room for the library function's own error
    for j in range(1, p):
        exact = mpmath.sin(mpmath.pi * j / p)
        err = abs(float((mpmath.mpf(s[j]) - exact) / exact))
        assert err <= 4 * 2.0 ** -53, (j, err)


def test_rader_tables_reproduce_the_dft(tables):
    modes, rec = tables
    rader = [n for n in SIZES if int(rec[("PLAN", n)][0]) == modes["rader"]]
    assert rader, "no Rader length among the sizes"
    rng = np.random.default_rng(9)
    for n in rader:
        p, N = n + 1, n
        pin = np.array(list(map(int, rec[("PIN", n)])))
        pout = np.array(list(map(int, rec[("POUT", n)])))
        g = int(pin[1])
        assert pin[0] == 1 and sorted(pin) == list(range(1, p))
        assert all(pow(g, (p - 1) // q, p) != 1 for q in range(2, p) if (p - 1) % q == 0 and _is_prime(q))
        assert all(pin[b] == pow(g, b, p) and (pout[b] * pin[b]) % p == 1 for b in range(N))
        bh = _hex(rec[("BHAT", n)])
        Bhat = bh[0::2] + 1j * bh[1::2]
        B = np.exp(-2j * np.pi * pout / p)
        assert np.allclose(Bhat, np.fft.fft(B) / N, rtol=0, atol=1e-15)
        # Rader: X_{g^{-c}} = x_0 + sum_b x_{g^b} B_{c-b}, computed as a circular
        # convolution through the length-N DFT with the printed kernel
        x = rng.standard_normal(p) + 1j * rng.standard_normal(p)
        a = x[pin]
        conv = np.fft.ifft(np.fft.fft(a) * Bhat * N)
        X = np.empty(p, dtype=complex)
        X[0] = x.sum()
        X[pout] = x[0] + conv
        assert np.allclose(X, np.fft.fft(x), rtol=0, atol=1e-12 * np.abs(x).sum())


@pytest.mark.parametrize("n,ns,delta,kappa", PIVOTS)
def test_thomas_pivots_solve_the_mode_systems(tables, n, ns, delta, kappa):
    from scipy.linalg import solve_banded
    _, rec = tables
    vals = rec[("PIV", n)]
    assert int(vals[0]) == ns
    r = _hex(vals[1:]).reshape(n, ns)
    rng = np.random.default_rng(n)
    for k in (1, 2, n // 2 + 1, n):
        d = -4 * delta + 2 * delta * np.cos(k * np.pi / (n + 1)) + kappa
        f = rng.standard_normal(ns)
        rk = r[k - 1]
        y = np.empty(ns)
        y[0] = rk[0] * f[0]
        for s in range(1, ns):
            y[s] = rk[s] * (f[s] - delta * y[s - 1])
        x = np.empty(ns)
        x[-1] = y[-1]
        for s in range(ns - 2, -1, -1):
            x[s] = y[s] - delta * rk[s] * x[s + 1]
        ab = np.zeros((3, ns))
        ab[0, 1:] = delta
        ab[1, :] = d
        ab[2, :-1] = delta
        want = solve_banded((1, 1), ab, f)
        assert np.allclose(x, want, rtol=1e-12, atol=1e-14 * np.abs(want).max()), (n, k)


def _sweep_matches_banded(r, mneg, delta, diag, rng, label):
    """The library's Thomas sweep (y_s = r_s (f_s - delta y_{s-1}), x_s = y_s + m_s x_{s+1},
    m_s = -delta r_s) with the printed pivots solves tridiag(delta, diag, delta) x = f as
    LAPACK's banded solver does."""
    from scipy.linalg import solve_banded
    ns = len(r)
    assert np.array_equal(mneg, -delta * r), label
    f = rng.standard_normal(ns)
    y = np.empty(ns)
    y[0] = r[0] * f[0]
    for s in range(1, ns):
        y[s] = r[s] * (f[s] - delta * y[s - 1])
    x = np.empty(ns)
    x[-1] = y[-1]
    for s in range(ns - 2, -1, -1):
        x[s] = y[s] + mneg[s] * x[s + 1]
    ab = np.zeros((3, ns))
    ab[0, 1:] = delta
    ab[1, :] = diag
    ab[2, :-1] = delta
    want = solve_banded((1, 1), ab, f)
    assert np.allclose(x, want, rtol=1e-12, atol=1e-14 * np.abs(want).max()), label


@pytest.mark.parametrize("case", range(len(DPIVOTS)))
def test_neumann_pivots_solve_the_mode_systems(tables, case):
    """Mode k of a line whose transform is the DCT-II has the eigenvalue mu_k of the
    cell-centred Neumann line operator (taken from the oracle, whose eigenpairs are
    pinned against that matrix): its sweep solves tridiag(delta, -2 delta + mu_k +
    kappa, delta), with the end row's extra term of a Neumann-sided arm."""
    from oracle.neumann import neumann_eigenvalues
    _, rec = tables
    nt, ns, delta, kappa, extra, end = DPIVOTS[case]
    v = _hex(rec[("DPIV", case)])
    r, m = v[:nt * ns].reshape(nt, ns), v[nt * ns:].reshape(nt, ns)
    mu = neumann_eigenvalues(nt, delta)
    rng = np.random.default_rng(case)
    for k in range(nt):
        diag = np.full(ns, -2 * delta + mu[k] + kappa)
        diag[0 if end == 0 else ns - 1] += extra
        _sweep_matches_banded(r[k], m[k], delta, diag, rng, (case, k))


@pytest.mark.parametrize("case", range(len(RPIVOTS)))
def test_periodic_pivots_solve_the_mode_systems(tables, case):
    """The same for periodic lines, with the circulant's eigenvalues mu_k from the
    oracle (mode k of the real-DFT coordinates, Re X_k or Im X_k, shares mu_k)."""
    from oracle.periodic import periodic_eigenvalues
    _, rec = tables
    nt, ns, delta, kappa = RPIVOTS[case]
    v = _hex(rec[("RPIV", case)])
    r, m = v[:nt * ns].reshape(nt, ns), v[nt * ns:].reshape(nt, ns)
    mu = periodic_eigenvalues(nt, delta)
    rng = np.random.default_rng(100 + case)
    for k in range(nt):
        _sweep_matches_banded(r[k], m[k], delta, np.full(ns, -2 * delta + mu[k] + kappa), rng, (case, k))


def _schur_term_matches(G, bs, n):
    """Every arm's R_ca A_a^{-1} R_ac, columns by sparse LU solves, against G on the
    centre's facing line; zero off that line."""
    # the centre's facing line of each arm, in the order of its line index
    # (centre row-major, x fastest; W/E face columns 0 / n-1, S/N face rows 0 / n-1)
    lines = {"W": [j * n for j in range(n)], "E": [j * n + n - 1 for j in range(n)],
             "S": list(range(n)), "N": [(n - 1) * n + i for i in range(n)]}
    scale = np.abs(G).max()
    for arm, idx in lines.items():
        M = np.empty((n, n))
        for j, cj in enumerate(idx):
            e = np.zeros(n * n)
            e[cj] = 1.0
            col = bs.R_c[arm] @ bs.block_solve(arm, bs.R_a[arm] @ e)
            M[:, j] = col[idx]
            rest = np.delete(col, idx)
            assert np.abs(rest).max() <= 1e-13 * scale  # the term lives on the facing line only
        err = np.abs(M - G).max() / scale
        assert err <= 1e-14, (arm, err)  # measured at most 5.4e-16 (Dirichlet and Neumann sides)


@pytest.mark.parametrize("case", range(len(CTABS)))
def test_interface_table_is_the_arms_exact_schur_term(tables, case):
    """The interface table behind the reduced Schur form (a2): for every arm of the
    cross, R_ca A_a^{-1} R_ac restricted to the centre's facing line, with A_a^{-1}
    a sparse LU of the oracle's arm block, equals G(i, j) = T(|i-j|) - H(i+j) built
    on the host from the arm's eigenvalues (Eq. "Schur_subeq" read as P2)."""
    from oracle.operator import assemble
    from oracle.schur import BlockSystem
    _, rec = tables
    n_s, kappa_s, *vals = rec[("CTAB", case)]
    n, kappa = int(n_s), float.fromhex(kappa_s)
    assert (n, kappa) == CTABS[case]
    _schur_term_matches(_hex(vals).reshape(n, n), BlockSystem(assemble("cross", n, kappa), "cross", n), n)


@pytest.mark.parametrize("case", range(len(CTABS)))
def test_neumann_interface_table_is_the_arms_exact_schur_term(tables, case):
    """The same for the cross whose arms have Neumann sides (P20, P21): the table
    built from the DCT-II eigenvalues and the arm's own pivots equals R_ca A_a^{-1}
    R_ac of the oracle's cell-centred Neumann-sided cross."""
    from oracle import neumann_cross as NC
    from oracle.schur import BlockSystem
    _, rec = tables
    n_s, kappa_s, *vals = rec[("CTABN", case)]
    n, kappa = int(n_s), float.fromhex(kappa_s)
    assert (n, kappa) == CTABS[case]
    bs = BlockSystem(NC.assemble(n, kappa), "cross", n, blocks=NC.block_ranges(n))
    _schur_term_matches(_hex(vals).reshape(n, n), bs, n)


@pytest.mark.parametrize("case", range(4))
def test_cluster_tables_are_the_scaled_thomas_pivots(tables, case):
    """The one-pass FP32 fast solve rewrites the LU recurrence of tridiag(delta, d_k,
    delta), u_s = d_k - delta^2 / u_{s-1}, for w_s = -u_s / delta - 1 (a sum of positive
    terms, accurate in the lowest modes where u_s is close to -2 delta).  Its host tables
    must therefore be sigma_k = 4 sin^2(k pi / 2p) - kappa / delta (40-digit values) and,
    at the first row s = r R of every CTA r, w_s = -1 / (delta r_s) - 1 from the
    reciprocal pivots r_s that the LAPACK test above pins -- each rounded once to
    binary32, so within an ulp of binary32."""
    _, rec = tables
    n_s, kappa_s, ok, R, *vals = rec[("CLUS", case)]
    n, kappa, R = int(n_s), float.fromhex(kappa_s), int(R)
    assert int(ok) == 1 and n % R == 0
    C, p = n // R, n + 1
    delta = float(p * p)
    v = _hex(vals)
    sigma, wseed, r = v[:n], v[n:n + C * n].reshape(C, n), v[n + C * n:].reshape(n, n)
    assert len(v) == n + C * n + n * n
    mpmath.mp.dps = 40
    s_ref = np.array([float(4 * mpmath.sin(k * mpmath.pi / (2 * p)) ** 2 - mpmath.mpf(kappa) / delta)
                      for k in range(1, n + 1)])
    f32 = np.float32
    assert np.all(np.abs(sigma - s_ref.astype(f32)) <= np.spacing(s_ref.astype(f32))), "sigma"
    w_ref = -1.0 / (delta * r[:, ::R].T) - 1.0  # [cta][k]
    assert np.all(np.abs(wseed - w_ref.astype(f32)) <= np.spacing(w_ref.astype(f32))), "w seeds"


def test_cluster_tables_only_for_the_kernels_lengths(tables):
    _, rec = tables
    assert rec[("CLUSNO", 0)] == ["0", "0"]


@pytest.mark.parametrize("nt", [8, 12, 256])
def test_dct_twiddles(tables, nt):
    """The DCT-II lines' tables (Makhoul's reordering on a complex FFT of length n):
    W[m] = e^{-2 pi i m/n} and post[k] = e^{-i pi k/(2n)}, interleaved (re, im), against
    40-digit values.  The angles are formed in floating point without folding, so each
    entry may carry the rounding of its angle a (up to |a| 2^-53, passed on with a
    derivative of at most 1) besides the function's own rounding: the bound is
    (1 + |a|) 2^-53 per entry (measured up to 4.4e-16 at n = 12, angles near 2 pi)."""
    _, rec = tables
    v = _hex(rec[("DCTW", nt)])
    W, post = v[:2 * nt], v[2 * nt:]
    assert len(post) == 2 * nt
    mpmath.mp.dps = 40
    u = 2.0 ** -53
    for m in range(nt):
        a = -2 * mpmath.pi * m / nt
        b = -mpmath.pi * m / (2 * nt)
        for got, want, ang in ((W[2 * m], mpmath.cos(a), a), (W[2 * m + 1], mpmath.sin(a), a),
                               (post[2 * m], mpmath.cos(b), b), (post[2 * m + 1], mpmath.sin(b), b)):
            assert abs(float(got - want)) <= (1 + abs(float(ang))) * u, (m, float(ang))
