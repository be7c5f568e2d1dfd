// Host-side tables and workspace carving shared by the domain API and the
// rectangle / box plans: a bump allocator over a caller's workspace, cos(pi m/d)
// with exact argument folding, the reciprocal Thomas pivots of the Dirichlet
// line operators, and the DST-I plan of a line length (radices of the Stockham
// FFT, Rader's permutations and kernel, the dense fallback).  Host code only.
#pragma once

#include <cmath>
#include <vector>

#include "fpg_dst.cuh"

namespace fpg {

// Bump allocator over the caller's workspace (256-byte aligned regions).  With
// base == nullptr it only measures.
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base((char*)b) {}
  void* take(size_t bytes) {
    used = (used + 255) & ~(size_t)255;
    void* p = base ? base + used : nullptr;
    used += bytes;
    return p;
  }
};

// Host tables in FP64 -------------------------------------------------------
inline double cos_pi_frac(long long num, long long den) {
  // cos(pi num / den) with exact folding to the first octant: the integer angle is
  // reduced to [0, pi/2] by symmetry, and past pi/4 the value is taken as the sine of
  // the complementary angle, so an entry near zero keeps its relative accuracy and
  // cos(pi/2) is exactly 0
  long long q = num % (2 * den);
  if (q < 0) q += 2 * den;
  if (q > den) q = 2 * den - q;                   // cos(2pi - x) = cos x
  double sign = 1.0;
  if (2 * q > den) { q = den - q; sign = -1.0; }  // cos(pi - x) = -cos x
  if (4 * q > den)                                // cos x = sin(pi/2 - x)
    return sign * std::sin(M_PI * (double)(den - 2 * q) / (double)(2 * den));
  return sign * std::cos(M_PI * (double)q / (double)den);
}

// Reciprocal Thomas pivots for tridiag(delta, d_k, delta) of length ns, all modes,
// into caller storage of n * ns doubles laid out [k][s], s fastest (one
// contiguous column per mode); d_k = -4 delta + 2 delta cos(k pi/(n+1)) + kappa.
inline void fill_pivots_into(int n, int ns, double delta, double kappa, double* r) {
  for (int k = 1; k <= n; ++k) {
    const double d = -4.0 * delta + 2.0 * delta * cos_pi_frac(k, n + 1) + kappa;
    double* rk = r + (size_t)(k - 1) * ns;
    double rp = 1.0 / d;
    rk[0] = rp;
    for (int s = 1; s < ns; ++s) {
      rp = 1.0 / (d - delta * delta * rp);
      rk[s] = rp;
    }
  }
}

inline void fill_pivots(int n, int ns, double delta, double kappa, std::vector<double>& r) {
  r.resize((size_t)ns * n);
  fill_pivots_into(n, ns, delta, kappa, r.data());
}


// DST plan for transform length n: radices of the Stockham FFT (4s, then a 2,
// then odd primes up to 43), Rader for a prime p whose p-1 factors that way,
// the dense fallback otherwise.
struct HostPlan {
  int mode = DST_DENSE, N = 0, nrad = 0, rad[kMaxRadices] = {0};
  std::vector<double> W, sinp, Bhat, dense;
  std::vector<int> pin, pout;
};

inline bool radices_for(int N, int* rad, int* nrad) {
  static const int odd[] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43};
  int m = N, twos = 0, cnt = 0;
  while (m % 2 == 0) { m /= 2; ++twos; }
  while (twos >= 2) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 4; twos -= 2; }
  if (twos == 1) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 2; }
  for (int q : odd) {
    while (m % q == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = q; m /= q; }
  }
  *nrad = cnt;
  return m == 1 && cnt > 0;
}

inline bool is_prime(int p) {
  if (p < 2) return false;
  for (int d = 2; (long long)d * d <= p; ++d) if (p % d == 0) return false;
  return true;
}

inline int primitive_root(int p) {
  // distinct prime factors of p - 1 (a 32-bit p - 1 has at most 9 of them);
  // fixed arrays, no heap, so the no-allocation entry point can call it
  int fs[32], nf = 0;
  int m = p - 1;
  for (int d = 2; (long long)d * d <= m; ++d) {
    if (m % d == 0) { fs[nf++] = d; while (m % d == 0) m /= d; }
  }
  if (m > 1) fs[nf++] = m;
  for (int g = 2; g < p; ++g) {
    bool ok = true;
    for (int i = 0; i < nf; ++i) {
      long long r = 1, b = g, e = (p - 1) / fs[i];
      while (e) { if (e & 1) r = r * b % p; b = b * b % p; e >>= 1; }
      if (r == 1) { ok = false; break; }
    }
    if (ok) return g;
  }
  return -1;
}

// exp(-2 pi i num/den) with exact folding of the argument
inline void cexp_neg(long long num, long long den, double* re, double* im) {
  *re = cos_pi_frac(2 * num, den);
  // sin(2 pi num/den) = cos(pi (4 num - den) / (2 den))
  *im = -cos_pi_frac(4 * num - den, 2 * den);
}

// Rader's tables for a prime p (N = p - 1), into caller storage: the input and
// output permutations pin[b] = g^b mod p and pout[b] = g^-b mod p for a
// primitive root g, and Bhat = DFT_N(B) / N (N complex values, re/im
// interleaved) with B_c = exp(-2 pi i g^-c / p).  No heap.
inline void rader_tables(int p, int* pin, int* pout, double* Bhat) {
  const int N = p - 1, g = primitive_root(p);
  long long ginv = 1;
  {  // g^{p-2} mod p
    long long b = g, e = p - 2;
    while (e) { if (e & 1) ginv = ginv * b % p; b = b * b % p; e >>= 1; }
  }
  long long a = 1, c = 1;
  for (int b = 0; b < N; ++b) {
    pin[b] = (int)a;
    pout[b] = (int)c;
    a = a * g % p;
    c = c * ginv % p;
  }
  for (int k = 0; k < N; ++k) {
    long double sr = 0, si = 0;
    for (int q = 0; q < N; ++q) {
      double br, bi, wr, wi;
      cexp_neg(pout[q], p, &br, &bi);
      cexp_neg((long long)q * k % N, N, &wr, &wi);
      sr += (long double)br * wr - (long double)bi * wi;
      si += (long double)br * wi + (long double)bi * wr;
    }
    Bhat[2 * k] = (double)(sr / N);
    Bhat[2 * k + 1] = (double)(si / N);
  }
}

inline HostPlan build_plan(int n) {
  HostPlan P;
  const int p = n + 1;
  P.sinp.resize(p);
  for (int j = 0; j < p; ++j) P.sinp[j] = cos_pi_frac(2 * j - p, 2 * p);  // sin(pi j/p) = cos(pi (j/p - 1/2))
  P.dense.resize(2 * p);
  for (int m = 0; m < 2 * p; ++m) P.dense[m] = cos_pi_frac(2 * m - p, 2 * p);
  int rad[kMaxRadices], nrad = 0;
  if (radices_for(p, rad, &nrad)) {
    P.mode = DST_STOCKHAM;
    P.N = p;
  } else if (is_prime(p) && radices_for(p - 1, rad, &nrad)) {
    P.mode = DST_RADER;
    P.N = p - 1;
  } else {
    P.mode = DST_DENSE;
    P.N = 1;
    nrad = 0;
  }
  P.nrad = nrad;
  for (int i = 0; i < nrad; ++i) P.rad[i] = rad[i];
  P.W.resize(2 * P.N);
  for (int m = 0; m < P.N; ++m) cexp_neg(m, P.N, &P.W[2 * m], &P.W[2 * m + 1]);
  if (P.mode == DST_RADER) {
    P.pin.resize(P.N);
    P.pout.resize(P.N);
    P.Bhat.resize(2 * P.N);
    rader_tables(p, P.pin.data(), P.pout.data(), P.Bhat.data());
  }
  return P;
}

// Radix plan only (sizes), no tables: used for workspace sizing.
inline HostPlan plan_shape(int n) {
  HostPlan P;
  const int p = n + 1;
  int rad[kMaxRadices], nrad = 0;
  if (radices_for(p, rad, &nrad)) { P.mode = DST_STOCKHAM; P.N = p; }
  else if (is_prime(p) && radices_for(p - 1, rad, &nrad)) { P.mode = DST_RADER; P.N = p - 1; }
  else { P.mode = DST_DENSE; P.N = 1; nrad = 0; }
  P.nrad = nrad;
  for (int i = 0; i < nrad; ++i) P.rad[i] = rad[i];
  return P;
}

// Host tables of the DCT-II lines: W[m] = e^{-2 pi i m/n}, post[k] = e^{-i pi k/(2n)}
// (interleaved re, im; n entries each).
inline void dct_tables(int n, std::vector<double>& W, std::vector<double>& post) {
  const double pi = 3.14159265358979323846;
  W.resize(2 * n);
  post.resize(2 * n);
  for (int i = 0; i < n; ++i) {
    const double a = 2.0 * pi * (double)i / n;
    W[2 * i] = std::cos(a);
    W[2 * i + 1] = -std::sin(a);
    const double b = pi * (double)i / (2.0 * n);
    post[2 * i] = std::cos(b);
    post[2 * i + 1] = -std::sin(b);
  }
}

// Reciprocal Thomas pivots r[k][s] and m = -delta r of the mode-k sweeps along
// s of a block with Neumann ends along t:  tridiag(delta, -2 delta + mu_k + kappa,
// delta), mu_k = -4 delta sin^2(k pi/(2n)), with `end_extra` added to the
// diagonal of row 0 (end = 0) or of row ns-1 (end = 1) -- -delta for a
// Dirichlet face half a cell beyond that row, 0 for a vertex-centred end.
inline void dct_pivots(int nt, int ns, double delta, double kappa, double end_extra, int end, std::vector<double>& r,
                std::vector<double>& m) {
  const double pi = 3.14159265358979323846;
  r.resize((size_t)nt * ns);
  m.resize((size_t)nt * ns);
  for (int k = 0; k < nt; ++k) {
    const double sk = std::sin(pi * (double)k / (2.0 * nt));
    const double d = -2.0 * delta - 4.0 * delta * sk * sk + kappa;
    double* rk = r.data() + (size_t)k * ns;
    double* mk = m.data() + (size_t)k * ns;
    double rp = 0.0;
    for (int s = 0; s < ns; ++s) {
      double ds = d;
      if ((end == 0 && s == 0) || (end == 1 && s == ns - 1)) ds += end_extra;
      rp = s == 0 ? 1.0 / ds : 1.0 / (ds - delta * delta * rp);
      rk[s] = rp;
      mk[s] = -delta * rp;
    }
  }
}

// Pivots of the periodic lines: mode m has mu_m = -4 delta sin^2(pi m/n), plain
// Dirichlet ends along s.
inline void rdft_pivots(int nt, int ns, double delta, double kappa, std::vector<double>& r, std::vector<double>& m) {
  const double pi = 3.14159265358979323846;
  r.resize((size_t)nt * ns);
  m.resize((size_t)nt * ns);
  for (int k = 0; k < nt; ++k) {
    const double sk = std::sin(pi * (double)k / nt);
    const double d = -2.0 * delta - 4.0 * delta * sk * sk + kappa;
    double* rk = r.data() + (size_t)k * ns;
    double* mk = m.data() + (size_t)k * ns;
    double rp = 0.0;
    for (int s = 0; s < ns; ++s) {
      rp = s == 0 ? 1.0 / d : 1.0 / (d - delta * delta * rp);
      rk[s] = rp;
      mk[s] = -delta * rp;
    }
  }
}

// Interface table of the reduced Schur form: c(m) = delta^2/(n+1) sum_k g_k cos(pi k m/(n+1)),
// m = 0..2n+1, with g_k = [T_k^{-1}]_{N,N} (N = n+1, the arm's sweep length) = last reciprocal pivot.
inline void fill_ctab(int n, double delta, const std::vector<double>& rpivA, std::vector<double>& c) {
  const int N = n + 1;
  c.resize(2 * n + 2);
  std::vector<double> g(n);
  for (int k = 1; k <= n; ++k) g[k - 1] = rpivA[(size_t)(k - 1) * N + N - 1];
  for (int m = 0; m < 2 * n + 2; ++m) {
    // compensated (Kahan) FP64 summation: exact to ~1 ulp of the sum
    double acc = 0.0, comp = 0.0;
    for (int k = 1; k <= n; ++k) {
      const double term = g[k - 1] * cos_pi_frac((long long)k * m, n + 1) - comp;
      const double t = acc + term;
      comp = (t - acc) - term;
      acc = t;
    }
    c[m] = acc * delta * delta / (double)(n + 1);
  }
  c.resize(4 * n + 2);
  for (int m = 0; m < 2 * n; ++m) c[2 * n + 2 + m] = c[m + 2];  // H(m) = T(m + 2)
}

// The same table for arms with Neumann sides (cell-centred, DCT-II basis
// u_k(j) = a_k cos(k pi (j + 1/2)/n), a_0^2 = 1/n, a_k^2 = 2/n): with g_k the
// interface entry of T_k^{-1} (the last reciprocal pivot when the far end is
// row 0), G_ij = sum_k g_k u_k(i) u_k(j) = T(|i-j|) + T(i+j+1),
// T(m) = delta^2/n (g_0/2 + sum_{k>=1} g_k cos(pi k m/n)); stored H(m) = -T(m+1).
inline void fill_ctab_dct(int n, double delta, const std::vector<double>& rpivA, std::vector<double>& c) {
  c.assign(4 * n + 2, 0.0);
  std::vector<double> g(n);
  for (int k = 0; k < n; ++k) g[k] = rpivA[(size_t)k * n + n - 1];
  for (int m = 0; m < 2 * n + 2; ++m) {
    double acc = 0.5 * g[0], comp = 0.0;
    for (int k = 1; k < n; ++k) {
      const double term = g[k] * cos_pi_frac((long long)k * m, n) - comp;
      const double t = acc + term;
      comp = (t - acc) - term;
      acc = t;
    }
    c[m] = acc * delta * delta / (double)n;
  }
  for (int m = 0; m < 2 * n; ++m) c[2 * n + 2 + m] = -c[m + 1];
}

// Lines (rows) per CTA of the one-pass FP32 cluster fast solve.
constexpr int kClusterRows = 32;

// Host tables of the cluster kernel for an n x n Dirichlet block (p = n + 1,
// 1/h^2 = delta), kappa: sigma[k-1] = 4 sin^2(k pi / 2p) - kappa / delta and,
// per CTA r of the cluster, the scaled pivot w at its first row s = r R,
// wseed[r][k-1], from the FP64 recurrence w_0 = 1 + sigma,
// w_s = sigma + w_{s-1} / (1 + w_{s-1}).  Returns false for lengths the kernel
// does not take.
inline bool fast_solve_cluster_tables(int n, double delta, double kappa, std::vector<float>& sigma,
                               std::vector<float>& wseed) {
  const int p = n + 1;
  if (p != 65 && p != 513) return false;
  const int R = kClusterRows, C = n / R;
  sigma.assign(n, 0.0f);
  wseed.assign((size_t)C * n, 0.0f);
  for (int k = 1; k <= n; ++k) {
    const double sh = cos_pi_frac(p - k, 2 * p);  // sin(k pi / 2p)
    const double sg = 4.0 * sh * sh - kappa / delta;
    sigma[k - 1] = (float)sg;
    double w = 1.0 + sg;
    for (int s = 0; s < n; ++s) {
      if (s % R == 0) wseed[(size_t)(s / R) * n + (k - 1)] = (float)w;
      w = sg + w / (1.0 + w);
    }
  }
  return true;
}

}  // namespace fpg
