// Fast solve on Neumann rectangles (Sec. 2.2, Eq. "submat_Neumann"): n_t x n_s
// blocks whose two edges across the transform axis t carry a zero normal
// derivative (the first and last line rows lose one delta) and whose edges
// across s are Dirichlet.  Along t the line operator is diagonalised by the
// DCT-II basis c_k(j) = cos(k pi (j - 1/2)/n_t), eigenvalues
// mu_k = -4 delta sin^2(k pi/(2 n_t)), k = 0..n_t-1 (the paper's Q_N, here in the
// form that diagonalises the matrix it prints).  Three launches per batch:
//   * forward DCT-II of every line (Makhoul's reordering: v_m = x_{2m},
//     v_{n-1-m} = x_{2m+1}; X_k = Re(e^{-i pi k/(2n)} V_k) with V = DFT_n(v)),
//     two real lines packed into one complex FFT of length n_t (the Stockham
//     engine of fpg_dst.cuh), into scratch[b][k][s];
//   * one Thomas solve per (block, mode): tridiag(delta, -2 delta + mu_k + kappa,
//     delta) along s (k_thomas_reg of the Dirichlet path, its own pivot tables);
//   * the inverse: V_k = e^{i pi k/(2n)} (X_k - i X_{n-k}) (X_n = 0), v = IDFT(V),
//     x_{2m} = v_m, x_{2m+1} = v_{n-1-m} -- the exact inverse of the forward map.
//
// Periodic rectangles (Sec. 2.2, Eq. "submat_Periodic"): periodic along t,
// Dirichlet across s.  The circulant line operator has mu_k = -4 delta sin^2(pi k/n_t)
// with mu_k = mu_{n-k}; the real eigenbasis pairs frequencies k and n-k (the
// paper's Q_P, a Hartley-type basis).  Here the same real modes are the real and
// imaginary parts of the line's DFT: mode m holds Re X_m for 2m <= n_t and
// Im X_m otherwise, each a real eigen-coordinate with eigenvalue mu_m.  Two real
// lines share one complex FFT forward and one inverse, with the Thomas solves of
// the DCT-II path in between.

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"

namespace fpg {

cudaError_t launch_thomas_any(int prec, void* scratch, int n, int ns, const void* rpiv, const void* mneg, int nblk,
                              const int* active, int nper_active, cudaStream_t st, int wpb);

namespace {

constexpr int kNmThreads = 256;

// Radices of the Stockham plan for length N: powers of two as 16s, then one 8,
// 4 or 2 (the power-of-two family); any other N as 4s, a 2 and odd primes to
// 13.  False when N has a prime factor above 13.
bool dct_radices(int N, int* rad, int* nrad) {
  static const int odd[] = {3, 5, 7, 11, 13};
  int m = N, cnt = 0;
  if (N >= 8 && (N & (N - 1)) == 0) {
    while (m % 16 == 0 && m > 16) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 16; m /= 16; }
    if (cnt >= kMaxRadices) return false;
    rad[cnt++] = m;  // 16, 8, 4 or 2 -- the last, largest-stride stage
    *nrad = cnt;
    return true;
  }
  while (m % 4 == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 4; m /= 4; }
  if (m % 2 == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 2; m /= 2; }
  for (int q : odd)
    while (m % q == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = q; m /= q; }
  *nrad = cnt;
  return m == 1 && cnt > 0;
}

int nm_pairs(int nt) {
  // two ping-pong complex buffers of Q line pairs plus two tables within ~100 KB
  long long q = (100 * 1024 - 32LL * nt) / (32LL * nt);
  if (q > 8) q = 8;
  if (q < 1) q = 1;
  return (int)q;
}

size_t nm_smem(int nt, int Q) { return sizeof(C2<double>) * ((size_t)2 * Q * nt + 2 * nt); }

__device__ __forceinline__ int makhoul_slot(int t, int nt) {
  // position of x_t in the reordered sequence v: v_m = x_{2m}, v_{n-1-m} = x_{2m+1}
  return (t & 1) == 0 ? t >> 1 : nt - 1 - (t >> 1);
}

// Forward DCT-II of the lines of a batch of blocks: element (t, s) of block b
// at in + (b / nper) rhs_stride + off[b % nper] + t st + s ss; 2Q lines per CTA,
// result X_k of line s at scratch[b][k][s].
template <int MAXR>
__global__ void __launch_bounds__(kNmThreads)
k_dct_fwd(const double* __restrict__ in, BatchDesc ib, LineLayout L, DstPlan pl, const C2<double>* __restrict__ Wg,
          const C2<double>* __restrict__ postg, double* __restrict__ scratch, int Q, const int* __restrict__ active,
          int nper_active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  const int nt = L.nt, ns = L.ns;
  C2<double>* b0 = reinterpret_cast<C2<double>*>(smem_raw);
  C2<double>* b1 = b0 + (size_t)Q * nt;
  C2<double>* W = b1 + (size_t)Q * nt;
  C2<double>* post = W + nt;
  double* b0d = reinterpret_cast<double*>(b0);
  const int s0 = blockIdx.x * 2 * Q, nl = min(2 * Q, ns - s0);
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    W[i] = Wg[i];
    post[i] = postg[i];
  }
  const double* src = in + (long long)(b / ib.nper) * ib.rhs_stride + ib.off[b % ib.nper];
  // line l = 2q + c goes to component c of packed sequence q, in Makhoul order
  if (L.st == 1) {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int l = i / nt, t = i - l * nt;
      b0d[2 * ((l >> 1) * nt + makhoul_slot(t, nt)) + (l & 1)] = l < nl ? src[t + (long long)(s0 + l) * L.ss] : 0.0;
    }
  } else {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int t = i / (2 * Q), l = i - t * (2 * Q);
      b0d[2 * ((l >> 1) * nt + makhoul_slot(t, nt)) + (l & 1)] =
          l < nl ? src[(long long)t * L.st + (long long)(s0 + l) * L.ss] : 0.0;
    }
  }
  __syncthreads();
  const C2<double>* Z = stockham_fft<double, MAXR>(pl, b0, b1, Q, nt, W);
  double* dst = scratch + (long long)b * nt * ns + s0;
  for (int i = threadIdx.x; i < Q * nt; i += blockDim.x) {
    const int k = i / Q, q = i - k * Q;  // q fastest: runs of 2Q rows per mode
    const C2<double> zk = Z[q * nt + k], zc = Z[q * nt + (k == 0 ? 0 : nt - k)];
    // the DFTs of the two packed real lines, then X_k = Re(e^{-i pi k/(2n)} V_k)
    const C2<double> va{0.5 * (zk.x + zc.x), 0.5 * (zk.y - zc.y)};
    const C2<double> vb{0.5 * (zk.y + zc.y), -0.5 * (zk.x - zc.x)};
    const C2<double> pk = post[k];
    const int la = 2 * q;
    if (la < nl) dst[(long long)k * ns + la] = pk.x * va.x - pk.y * va.y;
    if (la + 1 < nl) dst[(long long)k * ns + la + 1] = pk.x * vb.x - pk.y * vb.y;
  }
}

// Inverse of k_dct_fwd (x = DCT-II^{-1} X, i.e. X_0/n + (2/n) sum_k X_k cos(...)),
// written into the batch layout of `out`.
template <int MAXR>
__global__ void __launch_bounds__(kNmThreads)
k_dct_inv(const double* __restrict__ scratch, double* __restrict__ out, BatchDesc ob, LineLayout L, DstPlan pl,
          const C2<double>* __restrict__ Wg, const C2<double>* __restrict__ postg, int Q,
          const int* __restrict__ active, int nper_active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  const int nt = L.nt, ns = L.ns;
  C2<double>* b0 = reinterpret_cast<C2<double>*>(smem_raw);
  C2<double>* b1 = b0 + (size_t)Q * nt;
  C2<double>* W = b1 + (size_t)Q * nt;
  C2<double>* post = W + nt;
  double* X = reinterpret_cast<double*>(b1);  // [2Q][nt] spectra, staged
  const int s0 = blockIdx.x * 2 * Q, nl = min(2 * Q, ns - s0);
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    W[i] = Wg[i];
    post[i] = postg[i];
  }
  const double* src = scratch + (long long)b * nt * ns + s0;
  for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
    const int k = i / (2 * Q), l = i - k * (2 * Q);
    X[l * nt + k] = l < nl ? src[(long long)k * ns + l] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Q * nt; i += blockDim.x) {
    const int q = i / nt, k = i - q * nt;
    const double* xa = X + (2 * q) * nt;
    const double* xb = xa + nt;
    const double c = post[k].x, s = -post[k].y;  // e^{i pi k/(2n)} = (c, s)
    const double a0 = xa[k], a1 = k == 0 ? 0.0 : xa[nt - k];
    const double b0v = xb[k], b1v = k == 0 ? 0.0 : xb[nt - k];
    const C2<double> va{c * a0 + s * a1, s * a0 - c * a1};  // e^{i theta}(X_k - i X_{n-k})
    const C2<double> vb{c * b0v + s * b1v, s * b0v - c * b1v};
    // packed spectrum V^a + i V^b, conjugated: the inverse DFT as a forward one
    b0[i] = C2<double>{va.x - vb.y, -(va.y + vb.x)};
  }
  __syncthreads();
  const C2<double>* Z = stockham_fft<double, MAXR>(pl, b0, b1, Q, nt, W);
  const double inv = 1.0 / nt;
  double* dst = out + (long long)(b / ob.nper) * ob.rhs_stride + ob.off[b % ob.nper];
  // v = conj(Z) / n: line 2q is the real part, line 2q + 1 the imaginary part
  if (L.st == 1) {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int l = i / nt, t = i - l * nt;
      if (l >= nl) continue;
      const C2<double> zm = Z[(l >> 1) * nt + makhoul_slot(t, nt)];
      dst[t + (long long)(s0 + l) * L.ss] = (l & 1) == 0 ? zm.x * inv : -zm.y * inv;
    }
  } else {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int t = i / (2 * Q), l = i - t * (2 * Q);
      if (l >= nl) continue;
      const C2<double> zm = Z[(l >> 1) * nt + makhoul_slot(t, nt)];
      dst[(long long)t * L.st + (long long)(s0 + l) * L.ss] = (l & 1) == 0 ? zm.x * inv : -zm.y * inv;
    }
  }
}

// Forward real DFT of the lines of a batch of blocks (periodic along t): mode m
// of line s gets Re X_m (2m <= n) or Im X_m (2m > n), X = DFT_n(x), written to
// scratch[b][m][s].
template <int MAXR>
__global__ void __launch_bounds__(kNmThreads)
k_rdft_fwd(const double* __restrict__ in, BatchDesc ib, LineLayout L, DstPlan pl, const C2<double>* __restrict__ Wg,
           double* __restrict__ scratch, int Q, const int* __restrict__ active, int nper_active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  const int nt = L.nt, ns = L.ns;
  C2<double>* b0 = reinterpret_cast<C2<double>*>(smem_raw);
  C2<double>* b1 = b0 + (size_t)Q * nt;
  C2<double>* W = b1 + (size_t)Q * nt;
  double* b0d = reinterpret_cast<double*>(b0);
  const int s0 = blockIdx.x * 2 * Q, nl = min(2 * Q, ns - s0);
  for (int i = threadIdx.x; i < nt; i += blockDim.x) W[i] = Wg[i];
  const double* src = in + (long long)(b / ib.nper) * ib.rhs_stride + ib.off[b % ib.nper];
  if (L.st == 1) {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int l = i / nt, t = i - l * nt;
      b0d[2 * ((l >> 1) * nt + t) + (l & 1)] = l < nl ? src[t + (long long)(s0 + l) * L.ss] : 0.0;
    }
  } else {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int t = i / (2 * Q), l = i - t * (2 * Q);
      b0d[2 * ((l >> 1) * nt + t) + (l & 1)] = l < nl ? src[(long long)t * L.st + (long long)(s0 + l) * L.ss] : 0.0;
    }
  }
  __syncthreads();
  const C2<double>* Z = stockham_fft<double, MAXR>(pl, b0, b1, Q, nt, W);
  double* dst = scratch + (long long)b * nt * ns + s0;
  for (int i = threadIdx.x; i < Q * nt; i += blockDim.x) {
    const int k = i / Q, q = i - k * Q;
    const C2<double> zk = Z[q * nt + k], zc = Z[q * nt + (k == 0 ? 0 : nt - k)];
    const C2<double> va{0.5 * (zk.x + zc.x), 0.5 * (zk.y - zc.y)};   // DFT of line 2q at k
    const C2<double> vb{0.5 * (zk.y + zc.y), -0.5 * (zk.x - zc.x)};  // DFT of line 2q+1 at k
    const bool re = 2 * k <= nt;
    const int la = 2 * q;
    if (la < nl) dst[(long long)k * ns + la] = re ? va.x : va.y;
    if (la + 1 < nl) dst[(long long)k * ns + la + 1] = re ? vb.x : vb.y;
  }
}

// Inverse of k_rdft_fwd: rebuild each line's Hermitian spectrum from its real
// modes (Re X_k = Y_min(k,n-k); Im X_k = Y_k for 2k > n, -Y_{n-k} for 0 < 2k < n,
// 0 for k = 0 and 2k = n), x = IDFT(X), written into the batch layout of `out`.
template <int MAXR>
__global__ void __launch_bounds__(kNmThreads)
k_rdft_inv(const double* __restrict__ scratch, double* __restrict__ out, BatchDesc ob, LineLayout L, DstPlan pl,
           const C2<double>* __restrict__ Wg, int Q, const int* __restrict__ active, int nper_active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  const int nt = L.nt, ns = L.ns;
  C2<double>* b0 = reinterpret_cast<C2<double>*>(smem_raw);
  C2<double>* b1 = b0 + (size_t)Q * nt;
  C2<double>* W = b1 + (size_t)Q * nt;
  double* X = reinterpret_cast<double*>(b1);  // [2Q][nt] real modes, staged
  const int s0 = blockIdx.x * 2 * Q, nl = min(2 * Q, ns - s0);
  for (int i = threadIdx.x; i < nt; i += blockDim.x) W[i] = Wg[i];
  const double* src = scratch + (long long)b * nt * ns + s0;
  for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
    const int k = i / (2 * Q), l = i - k * (2 * Q);
    X[l * nt + k] = l < nl ? src[(long long)k * ns + l] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Q * nt; i += blockDim.x) {
    const int q = i / nt, k = i - q * nt;
    const double* ya = X + (2 * q) * nt;
    const double* yb = ya + nt;
    const int kr = 2 * k <= nt ? k : nt - k;
    const bool zero_im = k == 0 || 2 * k == nt;
    const double ra = ya[kr], rb = yb[kr];
    const double ia = zero_im ? 0.0 : (2 * k > nt ? ya[k] : -ya[nt - k]);
    const double ib = zero_im ? 0.0 : (2 * k > nt ? yb[k] : -yb[nt - k]);
    // packed spectrum A + i B, conjugated: the inverse DFT as a forward one
    b0[i] = C2<double>{ra - ib, -(ia + rb)};
  }
  __syncthreads();
  const C2<double>* Z = stockham_fft<double, MAXR>(pl, b0, b1, Q, nt, W);
  const double inv = 1.0 / nt;
  double* dst = out + (long long)(b / ob.nper) * ob.rhs_stride + ob.off[b % ob.nper];
  if (L.st == 1) {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int l = i / nt, t = i - l * nt;
      if (l >= nl) continue;
      const C2<double> zm = Z[(l >> 1) * nt + t];
      dst[t + (long long)(s0 + l) * L.ss] = (l & 1) == 0 ? zm.x * inv : -zm.y * inv;
    }
  } else {
    for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
      const int t = i / (2 * Q), l = i - t * (2 * Q);
      if (l >= nl) continue;
      const C2<double> zm = Z[(l >> 1) * nt + t];
      dst[(long long)t * L.st + (long long)(s0 + l) * L.ss] = (l & 1) == 0 ? zm.x * inv : -zm.y * inv;
    }
  }
}

template <int MAXR>
cudaError_t pd_launch(const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib, double* out,
                      BatchDesc ob, int nblk, double* scratch, const int* active, int nper_active, cudaStream_t st) {
  const int nt = L.nt;
  const int Q = nm_pairs(nt);
  const size_t smem = nm_smem(nt, Q);
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_rdft_fwd<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_rdft_inv<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  const C2<double>* W = reinterpret_cast<const C2<double>*>(tb.plan.W);
  const dim3 grid((L.ns + 2 * Q - 1) / (2 * Q), nblk);
  k_rdft_fwd<MAXR><<<grid, kNmThreads, smem, st>>>(in, ib, L, tb.plan, W, scratch, Q, active, nper_active);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_thomas_any(64, scratch, nt, L.ns, tb.rpiv, tb.mneg, nblk, active, nper_active, st, tb.mt);
  if (e != cudaSuccess) return e;
  k_rdft_inv<MAXR><<<grid, kNmThreads, smem, st>>>(scratch, out, ob, L, tb.plan, W, Q, active, nper_active);
  return cudaGetLastError();
}

template <int MAXR>
cudaError_t nm_launch(const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib, double* out,
                      BatchDesc ob, int nblk, double* scratch, const int* active, int nper_active, cudaStream_t st) {
  const int nt = L.nt;
  const int Q = nm_pairs(nt);
  const size_t smem = nm_smem(nt, Q);
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_dct_fwd<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dct_inv<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  const C2<double>* W = reinterpret_cast<const C2<double>*>(tb.plan.W);
  const C2<double>* post = reinterpret_cast<const C2<double>*>(tb.post);
  const dim3 grid((L.ns + 2 * Q - 1) / (2 * Q), nblk);
  k_dct_fwd<MAXR><<<grid, kNmThreads, smem, st>>>(in, ib, L, tb.plan, W, post, scratch, Q, active, nper_active);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_thomas_any(64, scratch, nt, L.ns, tb.rpiv, tb.mneg, nblk, active, nper_active, st, tb.mt);
  if (e != cudaSuccess) return e;
  k_dct_inv<MAXR><<<grid, kNmThreads, smem, st>>>(scratch, out, ob, L, tb.plan, W, post, Q, active, nper_active);
  return cudaGetLastError();
}

}  // namespace

// DCT-II plan of length n (Stockham, radices 4, 2 and odd primes to 13); false
// when n is odd or has another prime factor.  Tables are not touched.
bool dct_plan_shape(int n, DstPlan* pl) {
  *pl = DstPlan{};
  if (n < 2 || (n & 1) || n > 2048) return false;
  pl->n = n;
  pl->p = n;
  pl->mode = DST_STOCKHAM;
  pl->N = n;
  return dct_radices(n, pl->rad, &pl->nrad);
}

// Real-DFT plan of length n (periodic lines): any n >= 2 whose prime factors are
// at most 13, n <= 2048.
bool rdft_plan_shape(int n, DstPlan* pl) {
  *pl = DstPlan{};
  if (n < 2 || n > 2048) return false;
  pl->n = n;
  pl->p = n;
  pl->mode = DST_STOCKHAM;
  pl->N = n;
  return dct_radices(n, pl->rad, &pl->nrad);
}

cudaError_t launch_fast_solve_rdft(const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib,
                                   double* out, BatchDesc ob, int nblk, double* scratch, const int* active,
                                   int nper_active, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  switch (plan_maxr(tb.plan)) {
    case 16: return pd_launch<16>(tb, L, in, ib, out, ob, nblk, scratch, active, nper_active, st);
    case 5: return pd_launch<5>(tb, L, in, ib, out, ob, nblk, scratch, active, nper_active, st);
    default: return pd_launch<13>(tb, L, in, ib, out, ob, nblk, scratch, active, nper_active, st);
  }
}

cudaError_t launch_fast_solve_dct(const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib,
                                  double* out, BatchDesc ob, int nblk, double* scratch, const int* active,
                                  int nper_active, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  switch (plan_maxr(tb.plan)) {
    case 16: return nm_launch<16>(tb, L, in, ib, out, ob, nblk, scratch, active, nper_active, st);
    case 5: return nm_launch<5>(tb, L, in, ib, out, ob, nblk, scratch, active, nper_active, st);
    default: return nm_launch<13>(tb, L, in, ib, out, ob, nblk, scratch, active, nper_active, st);
  }
}

}  // namespace fpg
