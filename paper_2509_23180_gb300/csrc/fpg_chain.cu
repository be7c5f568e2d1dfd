// The chain of K crosses: several coupled blocks (Sec. 2.3-2.4).  2K - 1 unit
// squares in a row along x form the coupled set -- centres at even positions,
// links between them -- with arms W and E at the row's ends and S_i, N_i below
// and above centre i; every arm touches one block and is eliminated exactly,
// and the row is solved by flexible GMRES.  Its preconditioner is the row's own
// operator, one fast solve of the whole rectangle (transforms along y, sweeps of
// nxc rows along x), or on request the block diagonal of its squares (one fast
// solve per square); both run on the a1 kernels.
//
// Layout of one full vector (vertex-centred grid, h = 1/(n+1)): the coupled row
// as one rectangle of nxc = (2K-1)(n+1) - 1 columns by n rows (x fastest; each
// square owns the line it shares with the next), then W and E ((n+1) x n, x
// fastest, each owning the line it shares with the row), S_1..S_K and
// N_1..N_K (n x (n+1)).  Centre i's columns start at x0(i) = 2 i (n+1).
//
// The kernels here are the row-shaped counterparts of the cross's: the Schur
// matvec's stencil and interface terms, Alg. 1 steps 3 and 5, and the global
// operator K of the acceptance test.
#include <cuda_runtime.h>

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"

namespace fpg {

cudaError_t launch_residual_finalize(const double* part, int gmax, int cnt, int nrhs, double* out, double* fnorm_out,
                                     double rtol, double* tolabs, cudaStream_t st);

namespace {

constexpr int kChainThreads = 256;

template <typename Tz>
__device__ __forceinline__ double cld(const Tz* p, long long i) {
  return dl::convert<double>(p[i]);
}

__device__ __forceinline__ int chain_x0(const ChainGeom& G, int i) { return 2 * i * (G.n + 1); }

// Value of the row's line facing arm `slot` (0 W, 1 E, 2..K+1 S_i, K+2..2K+1 N_i), position q.
template <typename Tz>
__device__ __forceinline__ double chain_line(const Tz* z, const ChainGeom& G, int slot, int q) {
  const int n = G.n, nxc = G.nxc, K = G.K;
  if (slot == 0) return cld(z, (long long)q * nxc);
  if (slot == 1) return cld(z, (long long)q * nxc + nxc - 1);
  if (slot < 2 + K) return cld(z, chain_x0(G, slot - 2) + q);
  return cld(z, (long long)(n - 1) * nxc + chain_x0(G, slot - 2 - K) + q);
}

// a2 interface part: corr[r][slot][i] = sum_j (T(|i-j|) - H(i+j)) line_slot[j]
// (the reduced arm response; ctab = T[2n+2] then H[2n], the cross's table: the
// arms are the same blocks).  CTA: 32 outputs x 8 column groups, the group
// partials summed in group order.
template <typename Tz>
__global__ void __launch_bounds__(256)
k_chain_schur_lines(const Tz* __restrict__ z, long long zstride, ChainGeom G, const double* __restrict__ ctab,
                    double* __restrict__ corr, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = G.n, nslots = 2 * G.K + 2;
  double* line = reinterpret_cast<double*>(smem_raw);
  double* c = line + n;
  double* hk = c + 2 * n + 2;
  double* part = hk + 2 * n;
  const int r = blockIdx.y / nslots, slot = blockIdx.y % nslots;
  if (active != nullptr && !active[r]) return;
  const Tz* zr = z + (long long)r * zstride;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int q = tid; q < n; q += 256) line[q] = chain_line(zr, G, slot, q);
  for (int q = tid; q < 4 * n + 2; q += 256) c[q] = ctab[q];
  __syncthreads();
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int per = (n + 7) / 8;
  const int j0 = threadIdx.y * per, j1 = min(n, j0 + per);
  double acc = 0.0;
  if (i < n)
    for (int j = j0; j < j1; ++j) acc = fma(c[i > j ? i - j : j - i] - hk[i + j], line[j], acc);
  part[threadIdx.y * 32 + threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < n) {
    double s = part[threadIdx.x];
#pragma unroll
    for (int g = 1; g < 8; ++g) s += part[g * 32 + threadIdx.x];
    corr[((long long)r * nslots + slot) * n + i] = s;
  }
}

// a2 stencil part: w = A_row z - the interface terms on the lines next to the arms.
// One CTA per (row j, right-hand side), threads along the row: no index division.
template <typename Tz>
__global__ void __launch_bounds__(kChainThreads)
k_chain_stencil(const Tz* __restrict__ z, long long zstride, double* __restrict__ w, long long wstride, ChainGeom G,
                double delta, double kappa, const double* __restrict__ corr, const int* __restrict__ active) {
  const int r = blockIdx.y, j = blockIdx.x;
  if (active != nullptr && !active[r]) return;
  const int n = G.n, nxc = G.nxc, K = G.K, nslots = 2 * K + 2;
  const Tz* zr = z + (long long)r * zstride + (long long)j * nxc;
  double* wr = w + (long long)r * wstride + (long long)j * nxc;
  const double* cr = corr + (long long)r * nslots * n;
  const int period = 2 * (n + 1);
  for (int i = threadIdx.x; i < nxc; i += blockDim.x) {
    const double zc = cld(zr, i);
    const double s = stencil_sum(zc, i > 0 ? cld(zr, i - 1) : 0.0, i < nxc - 1 ? cld(zr, i + 1) : 0.0,
                                 j > 0 ? cld(zr, i - nxc) : 0.0, j < n - 1 ? cld(zr, i + nxc) : 0.0);
    double v = fma(delta, s, kappa * zc);
    if (i == 0) v -= cr[0 * n + j];
    if (i == nxc - 1) v -= cr[1 * n + j];
    if (j == 0 || j == n - 1) {
      const int a = i / period, q = i - a * period;
      if (q < n) v -= j == 0 ? cr[(2 + a) * n + q] : cr[(2 + K + a) * n + q];  // column under / over centre a (n >= 2)
    }
    wr[i] = v;
  }
}

// Alg. 1 step 3: f'_row = f_row - sum_a R_ca q_a, q_a in the arm blocks of `q`.
__global__ void __launch_bounds__(kChainThreads)
k_chain_reduce_rhs(const double* __restrict__ f, const double* __restrict__ q, long long ntot, ChainGeom G,
                   double delta, double* __restrict__ fc) {
  const int r = blockIdx.y;
  const int n = G.n, nxc = G.nxc, K = G.K;
  const double* fr = f + (long long)r * ntot;
  const double* qr = q + (long long)r * ntot;
  double* out = fc + (long long)r * nxc * n;
  const long long nc = (long long)nxc * n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / nxc), i = (int)(idx - (long long)j * nxc);
    double v = fr[idx];
    if (i == 0) v -= delta * qr[G.off[0] + (long long)j * (n + 1) + n];
    if (i == nxc - 1) v -= delta * qr[G.off[1] + (long long)j * (n + 1)];
    const int a = i / (2 * (n + 1)), c = i - chain_x0(G, a);
    if (c < n) {
      if (j == 0) v -= delta * qr[G.off[2 + a] + (long long)n * n + c];
      if (j == n - 1) v -= delta * qr[G.off[2 + K + a] + c];
    }
    out[idx] = v;
  }
}

// Alg. 1 step 5: out_a = f_a - R_ac u for every arm; the row's block of p gets u.
__global__ void __launch_bounds__(kChainThreads)
k_chain_arm_rhs(const double* __restrict__ f, const double* __restrict__ u, long long ntot, ChainGeom G,
                double delta, double* __restrict__ out, double* __restrict__ p) {
  const int r = blockIdx.y;
  const int n = G.n, nxc = G.nxc, K = G.K;
  const long long nc = (long long)nxc * n, na = (long long)n * (n + 1);
  const double* fr = f + (long long)r * ntot;
  const double* ur = u + (long long)r * nc;
  double* o = out + (long long)r * ntot;
  double* pr = p + (long long)r * ntot;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ntot;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nc) {
      pr[idx] = ur[idx];
      continue;
    }
    const int slot = (int)((idx - nc) / na);
    const long long li = idx - nc - (long long)slot * na;
    double v = fr[idx];
    if (slot < 2) {  // (n+1) x n
      const int j = (int)(li / (n + 1)), i = (int)(li - (long long)j * (n + 1));
      if (slot == 0 && i == n) v -= delta * ur[(long long)j * nxc];
      if (slot == 1 && i == 0) v -= delta * ur[(long long)j * nxc + nxc - 1];
    } else {         // n x (n+1)
      const int j = (int)(li / n), i = (int)(li - (long long)j * n);
      if (slot < 2 + K) {
        if (j == n) v -= delta * ur[chain_x0(G, slot - 2) + i];
      } else if (j == 0) {
        v -= delta * ur[(long long)(n - 1) * nxc + chain_x0(G, slot - 2 - K) + i];
      }
    }
    o[idx] = v;
  }
}

// Global operator (a7): value of the neighbour (di, dj) of local node (i, j) of
// block `blk` (-1 = the row, 0.. = arm slot); zero on the domain's edge.
__device__ __forceinline__ double chain_nb(const double* pr, const ChainGeom& G, int blk, int i, int j, int di,
                                           int dj) {
  const int n = G.n, nxc = G.nxc, K = G.K;
  const int ni = i + di, nj = j + dj;
  if (blk < 0) {
    if (ni >= 0 && ni < nxc && nj >= 0 && nj < n) return pr[(long long)nj * nxc + ni];
    if (ni < 0) return pr[G.off[0] + (long long)nj * (n + 1) + n];
    if (ni >= nxc) return pr[G.off[1] + (long long)nj * (n + 1)];
    const int a = ni / (2 * (n + 1)), c = ni - chain_x0(G, a);
    if (c >= n) return 0.0;  // below / above a link or a shared line: the edge
    return nj < 0 ? pr[G.off[2 + a] + (long long)n * n + c] : pr[G.off[2 + K + a] + c];
  }
  const long long off = G.off[blk];
  if (blk < 2) {  // (n+1) x n
    if (ni >= 0 && ni <= n && nj >= 0 && nj < n) return pr[off + (long long)nj * (n + 1) + ni];
    if (blk == 0 && ni == n + 1) return pr[(long long)nj * nxc];
    if (blk == 1 && ni == -1) return pr[(long long)nj * nxc + nxc - 1];
    return 0.0;
  }
  if (ni >= 0 && ni < n && nj >= 0 && nj <= n) return pr[off + (long long)nj * n + ni];
  if (blk < 2 + K) return nj == n + 1 ? pr[chain_x0(G, blk - 2) + ni] : 0.0;
  return nj == -1 ? pr[(long long)(n - 1) * nxc + chain_x0(G, blk - 2 - K) + ni] : 0.0;
}

// y = K p; with f != nullptr also partials of ||f - K p||^2 and ||f||^2.
__global__ void __launch_bounds__(kChainThreads)
k_chain_global_apply(const double* __restrict__ p, double* __restrict__ y, const double* __restrict__ f,
                     long long ntot, ChainGeom G, double delta, double kappa, double* __restrict__ part, int gmax,
                     int nrhs) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  const int n = G.n, nxc = G.nxc;
  const long long nc = (long long)nxc * n, na = (long long)n * (n + 1);
  const double* pr = p + (long long)r * ntot;
  double rr = 0.0, ff = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ntot;
       idx += (long long)gridDim.x * blockDim.x) {
    int blk, i, j;
    if (idx < nc) {
      blk = -1;
      j = (int)(idx / nxc);
      i = (int)(idx - (long long)j * nxc);
    } else {
      blk = (int)((idx - nc) / na);
      const long long li = idx - nc - (long long)blk * na;
      const int nx = blk < 2 ? n + 1 : n;
      j = (int)(li / nx);
      i = (int)(li - (long long)j * nx);
    }
    const double pc = pr[idx];
    const double s = stencil_sum(pc, chain_nb(pr, G, blk, i, j, -1, 0), chain_nb(pr, G, blk, i, j, 1, 0),
                                 chain_nb(pr, G, blk, i, j, 0, -1), chain_nb(pr, G, blk, i, j, 0, 1));
    const double kp = fma(delta, s, kappa * pc);
    if (y) y[(long long)r * ntot + idx] = kp;
    if (f) {
      const double fv = f[(long long)r * ntot + idx];
      const double d = fv - kp;
      rr = fma(d, d, rr);
      ff = fma(fv, fv, ff);
    }
  }
  if (f) {
    rr = block_sum(rr, red);
    ff = block_sum(ff, red);
    if (threadIdx.x == 0) {
      part[((long long)0 * nrhs + r) * gmax + blockIdx.x] = rr;
      part[((long long)1 * nrhs + r) * gmax + blockIdx.x] = ff;
    }
  }
}

}  // namespace

cudaError_t launch_chain_schur(const void* z, int zprec, long long zstride, const ChainGeom& G, const double* ctab,
                               double* corr, const int* active, int nrhs, cudaStream_t st) {
  const int n = G.n;
  dim3 grid((n + 31) / 32, nrhs * (2 * G.K + 2));
  const size_t smem = sizeof(double) * (5 * n + 2 + 256);
  static PerDeviceOnce attr_set;
  if (auto once = attr_set.first()) {
    cudaFuncSetAttribute(k_chain_schur_lines<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_chain_schur_lines<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  if (zprec == 64)
    k_chain_schur_lines<double><<<grid, dim3(32, 8), smem, st>>>((const double*)z, zstride, G, ctab, corr, active);
  else
    k_chain_schur_lines<float><<<grid, dim3(32, 8), smem, st>>>((const float*)z, zstride, G, ctab, corr, active);
  return cudaGetLastError();
}

cudaError_t launch_chain_stencil(const void* z, int zprec, long long zstride, double* w, long long wstride,
                                 const ChainGeom& G, double delta, double kappa, const double* corr,
                                 const int* active, int nrhs, int gx, cudaStream_t st) {
  (void)gx;
  dim3 grid(G.n, nrhs);
  if (zprec == 64)
    k_chain_stencil<double><<<grid, kChainThreads, 0, st>>>((const double*)z, zstride, w, wstride, G, delta, kappa,
                                                            corr, active);
  else
    k_chain_stencil<float><<<grid, kChainThreads, 0, st>>>((const float*)z, zstride, w, wstride, G, delta, kappa,
                                                           corr, active);
  return cudaGetLastError();
}

cudaError_t launch_chain_reduce_rhs(const double* f, const double* q, long long ntot, const ChainGeom& G,
                                    double delta, double* fc, int nrhs, int gx, cudaStream_t st) {
  k_chain_reduce_rhs<<<dim3(gx, nrhs), kChainThreads, 0, st>>>(f, q, ntot, G, delta, fc);
  return cudaGetLastError();
}

cudaError_t launch_chain_arm_rhs(const double* f, const double* u, long long ntot, const ChainGeom& G, double delta,
                                 double* out, double* p, int nrhs, int gx, cudaStream_t st) {
  k_chain_arm_rhs<<<dim3(gx, nrhs), kChainThreads, 0, st>>>(f, u, ntot, G, delta, out, p);
  return cudaGetLastError();
}

cudaError_t launch_chain_global_apply(const double* p, double* y, const double* f, long long ntot, const ChainGeom& G,
                                      double delta, double kappa, double* part, int gmax, int nrhs, int gx,
                                      double* rel_out, double* fnorm_out, double rtol, double* tolabs,
                                      cudaStream_t st) {
  k_chain_global_apply<<<dim3(gx, nrhs), kChainThreads, 0, st>>>(p, y, f, ntot, G, delta, kappa, part, gmax, nrhs);
  if (f) return launch_residual_finalize(part, gmax, gx, nrhs, rel_out, fnorm_out, rtol, tolabs, st);
  return cudaGetLastError();
}

}  // namespace fpg
