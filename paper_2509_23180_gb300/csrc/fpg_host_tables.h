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
  // cos(pi num / den) with exact folding to [0, pi/2]
  long long q = num % (2 * den);
  if (q < 0) q += 2 * den;
  if (q > den) q = 2 * den - q;                   // cos(2pi - x) = cos x
  double sign = 1.0;
  if (2 * q > den) { q = den - q; sign = -1.0; }  // cos(pi - x) = -cos x
  return sign * std::cos(M_PI * (double)q / (double)den);
}

// Reciprocal Thomas pivots for tridiag(delta, d_k, delta) of length ns, all modes:
// r[s][k-1], d_k = -4 delta + 2 delta cos(k pi/(n+1)) + kappa.
inline void fill_pivots(int n, int ns, double delta, double kappa, std::vector<double>& r) {
  r.resize((size_t)ns * n);  // [k][s], s fastest (one contiguous column per mode)
  for (int k = 1; k <= n; ++k) {
    const double d = -4.0 * delta + 2.0 * delta * cos_pi_frac(k, n + 1) + kappa;
    double* rk = r.data() + (size_t)(k - 1) * ns;
    double rp = 1.0 / d;
    rk[0] = rp;
    for (int s = 1; s < ns; ++s) {
      rp = 1.0 / (d - delta * delta * rp);
      rk[s] = rp;
    }
  }
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
  std::vector<int> fs;
  int m = p - 1;
  for (int d = 2; (long long)d * d <= m; ++d) {
    if (m % d == 0) { fs.push_back(d); while (m % d == 0) m /= d; }
  }
  if (m > 1) fs.push_back(m);
  for (int g = 2; g < p; ++g) {
    bool ok = true;
    for (int q : fs) {
      long long r = 1, b = g, e = (p - 1) / q;
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
    const int N = P.N, g = primitive_root(p);
    long long ginv = 1;
    {  // g^{p-2} mod p
      long long b = g, e = p - 2;
      while (e) { if (e & 1) ginv = ginv * b % p; b = b * b % p; e >>= 1; }
    }
    P.pin.resize(N);
    P.pout.resize(N);
    long long a = 1, c = 1;
    for (int b = 0; b < N; ++b) {
      P.pin[b] = (int)a;
      P.pout[b] = (int)c;
      a = a * g % p;
      c = c * ginv % p;
    }
    // Bhat = DFT_N(B) / N with B_c = exp(-2 pi i g^{-c} / p)
    std::vector<double> Br(N), Bi(N);
    for (int q = 0; q < N; ++q) cexp_neg(P.pout[q], p, &Br[q], &Bi[q]);
    P.Bhat.resize(2 * N);
    for (int k = 0; k < N; ++k) {
      long double sr = 0, si = 0;
      for (int q = 0; q < N; ++q) {
        double wr, wi;
        cexp_neg((long long)q * k % N, N, &wr, &wi);
        sr += (long double)Br[q] * wr - (long double)Bi[q] * wi;
        si += (long double)Br[q] * wi + (long double)Bi[q] * wr;
      }
      P.Bhat[2 * k] = (double)(sr / N);
      P.Bhat[2 * k + 1] = (double)(si / N);
    }
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

}  // namespace fpg
