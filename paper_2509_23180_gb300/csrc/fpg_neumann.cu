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
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fpg_internal.cuh"

namespace fpg {

void record_message(const char* msg);
cudaError_t launch_thomas_any(int prec, void* scratch, int n, int ns, const void* rpiv, const void* mneg, int nblk,
                              cudaStream_t st);

namespace {

constexpr int kNmThreads = 256;

// Radices of the Stockham plan for length N (4, 2 and odd primes to 13); false
// when N has another factor.
bool dct_radices(int N, int* rad, int* nrad) {
  static const int odd[] = {3, 5, 7, 11, 13};
  int m = N, cnt = 0;
  while (m % 4 == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 4; m /= 4; }
  if (m % 2 == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = 2; m /= 2; }
  for (int q : odd)
    while (m % q == 0) { if (cnt >= kMaxRadices) return false; rad[cnt++] = q; m /= q; }
  *nrad = cnt;
  return m == 1 && cnt > 0;
}

struct NmLayout {  // byte offsets in the caller's workspace
  size_t W, post, rpiv, mneg, scratch, total;
};

NmLayout nm_layout(int nt, int ns, int nvec) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  NmLayout L{};
  size_t o = 0;
  L.W = o;       o = al(o + sizeof(double) * 2 * nt);
  L.post = o;    o = al(o + sizeof(double) * 2 * nt);
  L.rpiv = o;    o = al(o + sizeof(double) * (size_t)nt * ns);
  L.mneg = o;    o = al(o + sizeof(double) * (size_t)nt * ns);
  L.scratch = o; o = al(o + sizeof(double) * (size_t)nvec * nt * ns);
  L.total = o;
  return L;
}

int nm_pairs(int nt) {
  // two ping-pong complex buffers of Q line pairs plus two tables within ~100 KB
  long long q = (100 * 1024 - 32LL * nt) / (32LL * nt);
  if (q > 8) q = 8;
  if (q < 1) q = 1;
  return (int)q;
}

size_t nm_smem(int nt, int Q) { return sizeof(C2<double>) * ((size_t)2 * Q * nt + 2 * nt); }

template <int MAXR>
__global__ void __launch_bounds__(kNmThreads)
k_dct_fwd(const double* __restrict__ v, double* __restrict__ scratch, int nt, int ns, DstPlan pl,
          const C2<double>* __restrict__ Wg, const C2<double>* __restrict__ postg, int Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<double>* b0 = reinterpret_cast<C2<double>*>(smem_raw);
  C2<double>* b1 = b0 + (size_t)Q * nt;
  C2<double>* W = b1 + (size_t)Q * nt;
  C2<double>* post = W + nt;
  const int b = blockIdx.y, s0 = blockIdx.x * 2 * Q, nl = min(2 * Q, ns - s0);
  const int half = nt / 2;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    W[i] = Wg[i];
    post[i] = postg[i];
  }
  const double* src = v + (long long)b * nt * ns;
  for (int i = threadIdx.x; i < Q * nt; i += blockDim.x) {
    const int q = i / nt, m = i - q * nt;
    const int t = m < half ? 2 * m : 2 * (nt - 1 - m) + 1;  // Makhoul reordering
    const int la = 2 * q, lb = la + 1;
    const double a = la < nl ? src[(long long)(s0 + la) * nt + t] : 0.0;
    const double c = lb < nl ? src[(long long)(s0 + lb) * nt + t] : 0.0;
    b0[i] = C2<double>{a, c};
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

template <int MAXR>
__global__ void __launch_bounds__(kNmThreads)
k_dct_inv(const double* __restrict__ scratch, double* __restrict__ z, int nt, int ns, DstPlan pl,
          const C2<double>* __restrict__ Wg, const C2<double>* __restrict__ postg, int Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<double>* b0 = reinterpret_cast<C2<double>*>(smem_raw);
  C2<double>* b1 = b0 + (size_t)Q * nt;
  C2<double>* W = b1 + (size_t)Q * nt;
  C2<double>* post = W + nt;
  double* X = reinterpret_cast<double*>(b1);  // [2Q][nt] spectra, staged
  const int b = blockIdx.y, s0 = blockIdx.x * 2 * Q, nl = min(2 * Q, ns - s0);
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
  double* dst = z + (long long)b * nt * ns;
  for (int i = threadIdx.x; i < 2 * Q * nt; i += blockDim.x) {
    const int l = i / nt, t = i - l * nt;
    if (l >= nl) continue;
    const int m = (t & 1) == 0 ? t / 2 : nt - 1 - (t - 1) / 2;
    const C2<double> zm = Z[(l >> 1) * nt + m];
    // v = conj(Z) / n: line a is the real part, line b the imaginary part
    dst[(long long)(s0 + l) * nt + t] = (l & 1) == 0 ? zm.x * inv : -zm.y * inv;
  }
}

template <int MAXR>
cudaError_t nm_launch(const double* v, double* z, double* scratch, int nt, int ns, const DstPlan& pl,
                      const C2<double>* W, const C2<double>* post, const double* rpiv, const double* mneg, int nvec,
                      cudaStream_t st) {
  const int Q = nm_pairs(nt);
  const size_t smem = nm_smem(nt, Q);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dct_fwd<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dct_inv<MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const dim3 grid((ns + 2 * Q - 1) / (2 * Q), nvec);
  k_dct_fwd<MAXR><<<grid, kNmThreads, smem, st>>>(v, scratch, nt, ns, pl, W, post, Q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_thomas_any(64, scratch, nt, ns, rpiv, mneg, nvec, st);
  if (e != cudaSuccess) return e;
  k_dct_inv<MAXR><<<grid, kNmThreads, smem, st>>>(scratch, z, nt, ns, pl, W, post, Q);
  return cudaGetLastError();
}

}  // namespace
}  // namespace fpg

extern "C" fpg_status fpg_neumann_workspace_bytes(int32_t nt, int32_t ns, int32_t nvec, size_t* bytes) {
  if (!bytes || nt < 2 || (nt & 1) || ns < 1 || nvec < 1 || nt > 4096 || ns > 4096) return FPG_EINVAL;
  *bytes = fpg::nm_layout(nt, ns, nvec).total;
  return FPG_OK;
}

extern "C" fpg_status fpg_neumann_solve(int32_t nt, int32_t ns, double h, double kappa, const double* v, double* z,
                                        int32_t nvec, void* workspace, size_t bytes, void* stream) {
  using namespace fpg;
  if (!v || !z || !workspace || nt < 2 || (nt & 1) || ns < 1 || nvec < 1 || nt > 4096 || ns > 4096 ||
      !(h > 0.0) || !(kappa <= 0.0)) {
    record_message("fpg_neumann_solve: bad argument (n_t even >= 2, n_s >= 1, h > 0, kappa <= 0, pointers)");
    return FPG_EINVAL;
  }
  const NmLayout L = nm_layout(nt, ns, nvec);
  if (bytes < L.total) return FPG_ENOMEM;
  DstPlan pl{};
  pl.n = nt;
  pl.p = nt;
  pl.mode = DST_STOCKHAM;
  pl.N = nt;
  if (!dct_radices(nt, pl.rad, &pl.nrad) || plan_maxr(pl) > 13) {
    record_message("fpg_neumann_solve: n_t has a prime factor above 13");
    return FPG_EUNSUPPORTED;
  }
  // tables: w_n^m, e^{-i pi k/(2n)}, and the reciprocal Thomas pivots of
  // tridiag(delta, -2 delta + mu_k + kappa, delta) along s, laid out [k][s]
  const double delta = 1.0 / (h * h);
  const double pi = 3.14159265358979323846;
  std::vector<double> W(2 * nt), post(2 * nt), r((size_t)nt * ns), m((size_t)nt * ns);
  for (int i = 0; i < nt; ++i) {
    const double a = 2.0 * pi * (double)i / nt;
    W[2 * i] = std::cos(a);
    W[2 * i + 1] = -std::sin(a);
    const double b = pi * (double)i / (2.0 * nt);
    post[2 * i] = std::cos(b);
    post[2 * i + 1] = -std::sin(b);
  }
  for (int k = 0; k < nt; ++k) {
    const double sk = std::sin(pi * (double)k / (2.0 * nt));
    const double d = -2.0 * delta - 4.0 * delta * sk * sk + kappa;
    double rp = 1.0 / d;
    double* rk = r.data() + (size_t)k * ns;
    double* mk = m.data() + (size_t)k * ns;
    rk[0] = rp;
    mk[0] = -delta * rp;
    for (int s = 1; s < ns; ++s) {
      rp = 1.0 / (d - delta * delta * rp);
      rk[s] = rp;
      mk[s] = -delta * rp;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = static_cast<unsigned char*>(workspace);
  // pageable sources: each copy has finished reading its host buffer on return
  cudaError_t e = cudaMemcpyAsync(base + L.W, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + L.post, post.data(), sizeof(double) * post.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + L.rpiv, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + L.mneg, m.data(), sizeof(double) * m.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    pl.W = base + L.W;
    const C2<double>* Wd = reinterpret_cast<const C2<double>*>(base + L.W);
    const C2<double>* Pd = reinterpret_cast<const C2<double>*>(base + L.post);
    double* scratch = reinterpret_cast<double*>(base + L.scratch);
    const double* rd = reinterpret_cast<const double*>(base + L.rpiv);
    const double* md = reinterpret_cast<const double*>(base + L.mneg);
    e = plan_maxr(pl) <= 5 ? nm_launch<5>(v, z, scratch, nt, ns, pl, Wd, Pd, rd, md, nvec, st)
                           : nm_launch<13>(v, z, scratch, nt, ns, pl, Wd, Pd, rd, md, nvec, st);
  }
  if (e != cudaSuccess) {
    record_cuda_error(e, "fpg_neumann_solve");
    return FPG_ECUDA;
  }
  return FPG_OK;
}
