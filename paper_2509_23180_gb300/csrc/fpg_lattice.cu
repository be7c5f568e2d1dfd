// General concatenated geometry (FPG_GEOM_LATTICE): any edge-connected set of
// unit squares of an 8 x 8 grid, several coupled blocks in any arrangement
// (Sec. 2.3-2.4 and the rule after Alg. "fft_dd_solver": a sub-domain adjacent
// to only one other is independent and eliminated exactly; the others are
// coupled and solved together by GMRES).
//
// Partition of the unknowns (vertex-centred grid, m = n + 1 points per unit):
//   * coupled squares (two or more edge neighbours; of a lone pair the first):
//     their n x n interior points;
//   * links: the grid line shared by two coupled squares, n points;
//   * junctions: a lattice vertex with all four squares around it, one point;
//   * independent squares (one neighbour): interior plus the shared line,
//     (n+1) x n or n x (n+1) -- the arms of the cross, in any orientation.
// Block order: the coupled set first (squares in bit order, the links across
// vertical edges then across horizontal edges, each by (j, i), the junctions by
// (Y, X)), then the independent squares in bit order.  The coupled set is the
// Krylov vector: a prefix of the global vector.
//
// On the device the coupled set's operator is applied through a neighbour
// table (four indices per point) and the independent squares' Schur terms
// through the reduced interface form of the cross (Toeplitz-minus-Hankel table
// of the arm's sweep), one "face" per independent square.  The preconditioner
// is the block diagonal of the coupled set's parts: the fast solve of every
// coupled square (the centre's DST/Thomas engine, batched), a Thomas solve of
// every link's own tridiagonal operator tridiag(delta, -4 delta + kappa, delta)
// and the inverse diagonal of every junction.
#include <cuda_runtime.h>

#include <vector>

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"
#include "fpg_lattice_host.h"

namespace fpg {

// ---------------------------------------------------------------------------
// Kernels.  r = blockIdx.y is the right-hand side; inactive ones are skipped.
namespace {

constexpr int kThreads = 256;

template <typename Tz>
__device__ __forceinline__ double ldz(const Tz* p, long long i) {
  return dl::convert<double>(p[i]);  // integer-pipe widening for an FP32 basis
}

// a2, interface part: corr[r][f][i] = sum_j (T(|i-j|) - H(i+j)) line_f[j], the
// exact response R_ca A_a^{-1} R_ac of independent square a on the boundary
// line of its coupled neighbour (face f = (offset of that square, side)).
template <typename Tz>
__global__ void __launch_bounds__(256)
k_lat_faces(const Tz* __restrict__ z, long long zstride, const int2* __restrict__ faces, int nfaces, int n,
            const double* __restrict__ ctab, double* __restrict__ corr, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* line = reinterpret_cast<double*>(smem_raw);
  double* c = line + n;
  double* hk = c + 2 * n + 2;
  double* part = hk + 2 * n;  // [8][32]
  const int r = blockIdx.y / nfaces, f = blockIdx.y % nfaces;
  if (active != nullptr && !active[r]) return;
  const int2 fc = faces[f];
  const Tz* zr = z + (long long)r * zstride + fc.x;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int q = tid; q < n; q += 256) {
    long long at;
    switch (fc.y) {
      case 0: at = (long long)q * n; break;
      case 1: at = (long long)q * n + n - 1; break;
      case 2: at = q; break;
      default: at = (long long)(n - 1) * n + q; break;
    }
    line[q] = ldz(zr, at);
  }
  for (int q = tid; q < 4 * n + 2; q += 256) c[q] = ctab[q];
  __syncthreads();
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int per = (n + 7) / 8;
  const int j0 = threadIdx.y * per, j1 = min(n, j0 + per);
  double acc = 0.0;
  if (i < n) {
    for (int j = j0; j < j1; ++j) {
      const int d = i > j ? i - j : j - i;
      acc = fma(c[d] - hk[i + j], line[j], acc);
    }
  }
  part[threadIdx.y * 32 + threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < n) {
    double sum = part[threadIdx.x];
#pragma unroll
    for (int g = 1; g < 8; ++g) sum += part[g * 32 + threadIdx.x];
    corr[((long long)r * nfaces + f) * n + i] = sum;
  }
}

// a2: w = A_c z - (interface corrections), A_c the coupled set's own 5-point
// operator (neighbours outside the coupled set count as zero), in the
// difference form of the stencil.
template <typename Tz>
__global__ void __launch_bounds__(kThreads)
k_lat_stencil(const Tz* __restrict__ z, long long zstride, double* __restrict__ w, long long wstride, long long nc,
              const int4* __restrict__ nbr, const int2* __restrict__ cf, const double* __restrict__ corr,
              long long corr_stride, double delta, double kappa, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const Tz* zr = z + (long long)r * zstride;
  double* wr = w + (long long)r * wstride;
  const double* cr = corr + (long long)r * corr_stride;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
    const int4 q = nbr[i];
    const double zc = ldz(zr, i);
    const double s = stencil_sum(zc, q.x >= 0 ? ldz(zr, q.x) : 0.0, q.y >= 0 ? ldz(zr, q.y) : 0.0,
                                 q.z >= 0 ? ldz(zr, q.z) : 0.0, q.w >= 0 ? ldz(zr, q.w) : 0.0);
    double v = fma(delta, s, kappa * zc);
    const int2 c = cf[i];
    if (c.x >= 0) v -= cr[c.x];
    if (c.y >= 0) v -= cr[c.y];
    wr[i] = v;
  }
}

// Preconditioner on the links and junctions (the coupled squares go through the
// fast solve): each link's own tridiag(delta, d0, delta), d0 = -4 delta + kappa,
// by a Thomas sweep with the reciprocal pivots lpiv (one thread per link), each
// junction by 1 / d0.
template <typename Tz>
__global__ void __launch_bounds__(kThreads)
k_lat_skeleton(const double* __restrict__ v, Tz* __restrict__ z, long long stride, long long link_base, int nlinks,
               long long junc_base, int njunc, int n, const double* __restrict__ lpiv, double delta, double d0,
               const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const double* vr = v + (long long)r * stride;
  Tz* zr = z + (long long)r * stride;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nlinks) {
    const long long o = link_base + (long long)t * n;
    double y = 0.0;
    for (int s = 0; s < n; ++s) {  // forward: y_s = r_s (f_s - delta y_{s-1})
      y = lpiv[s] * fma(-delta, y, vr[o + s]);
      zr[o + s] = (Tz)y;
    }
    double x = 0.0;
    for (int s = n - 1; s >= 0; --s) {  // back: x_s = y_s - delta r_s x_{s+1}
      x = fma(-delta * lpiv[s], x, dl::convert<double>(zr[o + s]));
      zr[o + s] = (Tz)x;
    }
  } else if (t < nlinks + njunc) {
    const long long o = junc_base + (t - nlinks);
    zr[o] = (Tz)(vr[o] / d0);
  }
}

// Alg. 1 step 3: f'_c = f_c - sum R_ca q_a (the coupled set is the prefix of f).
__global__ void __launch_bounds__(kThreads)
k_lat_reduce_rhs(const double* __restrict__ f, const double* __restrict__ q, long long ntot, long long nc,
                 const int2* __restrict__ anb, double delta, double* __restrict__ fc) {
  const int r = blockIdx.y;
  const double* fr = f + (long long)r * ntot;
  const double* qr = q + (long long)r * ntot;
  double* o = fc + (long long)r * nc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
    const int2 a = anb[i];
    double v = fr[i];
    if (a.x >= 0) v -= delta * qr[a.x];
    if (a.y >= 0) v -= delta * qr[a.y];
    o[i] = v;
  }
}

// Alg. 1 steps 5-6: p_c = u; for the independent squares out = f - R_ac p_c.
__global__ void __launch_bounds__(kThreads)
k_lat_arm_rhs(const double* __restrict__ f, const double* __restrict__ u, long long ntot, long long nc,
              const int* __restrict__ gcn, double delta, double* __restrict__ out, double* __restrict__ p) {
  const int r = blockIdx.y;
  const double* fr = f + (long long)r * ntot;
  const double* ur = u + (long long)r * nc;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ntot; g += (long long)gridDim.x * blockDim.x) {
    if (g < nc) {
      p[(long long)r * ntot + g] = ur[g];
    } else {
      const int c = gcn[g];
      out[(long long)r * ntot + g] = c >= 0 ? fr[g] - delta * ur[c] : fr[g];
    }
  }
}

// a7: y = K p (optional) and partial sums of ||f - K p||^2 and ||f||^2.
__global__ void __launch_bounds__(kThreads)
k_lat_global(const double* __restrict__ p, double* __restrict__ y, const double* __restrict__ f, long long ntot,
             const int4* __restrict__ gnbr, double delta, double kappa, double* __restrict__ part, int gmax, int nrhs) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  const double* pr = p + (long long)r * ntot;
  double rr = 0.0, ff = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ntot; g += (long long)gridDim.x * blockDim.x) {
    const int4 q = gnbr[g];
    const double pc = pr[g];
    const double s = stencil_sum(pc, q.x >= 0 ? pr[q.x] : 0.0, q.y >= 0 ? pr[q.y] : 0.0, q.z >= 0 ? pr[q.z] : 0.0,
                                 q.w >= 0 ? pr[q.w] : 0.0);
    const double kp = fma(delta, s, kappa * pc);
    if (y) y[(long long)r * ntot + g] = kp;
    if (f) {
      const double fv = f[(long long)r * ntot + g];
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

cudaError_t launch_residual_finalize(const double* part, int gmax, int cnt, int nrhs, double* out, double* fnorm_out,
                                     double rtol, double* tolabs, cudaStream_t st);

cudaError_t launch_lattice_schur(const void* z, int zprec, long long zstride, double* w, long long wstride,
                                 const LatticeDev& t, int n, double delta, double kappa, const double* ctab,
                                 double* corr, const int* active, int nrhs, int gx, cudaStream_t st) {
  if (t.nfaces > 0) {
    const size_t smem = sizeof(double) * (n + 4 * n + 2 + 256);
    const dim3 grid((n + 31) / 32, nrhs * t.nfaces), block(32, 8);
    static PerDeviceOnce attr;
    if (auto once = attr.first()) {
      cudaFuncSetAttribute(k_lat_faces<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(k_lat_faces<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    if (zprec == 64)
      k_lat_faces<double><<<grid, block, smem, st>>>((const double*)z, zstride, t.faces, t.nfaces, n, ctab, corr,
                                                     active);
    else
      k_lat_faces<float><<<grid, block, smem, st>>>((const float*)z, zstride, t.faces, t.nfaces, n, ctab, corr,
                                                    active);
  }
  const dim3 grid(gx, nrhs);
  const long long cs = (long long)t.nfaces * n;
  if (zprec == 64)
    k_lat_stencil<double><<<grid, kThreads, 0, st>>>((const double*)z, zstride, w, wstride, t.nc, t.nbr, t.cf, corr,
                                                     cs, delta, kappa, active);
  else
    k_lat_stencil<float><<<grid, kThreads, 0, st>>>((const float*)z, zstride, w, wstride, t.nc, t.nbr, t.cf, corr,
                                                    cs, delta, kappa, active);
  return cudaGetLastError();
}

cudaError_t launch_lattice_skeleton(const double* v, void* z, int zprec, const LatticeDev& t, int n, double delta,
                                    double kappa, const int* active, int nrhs, cudaStream_t st) {
  const int items = t.nlinks + t.njunc;
  if (items == 0) return cudaSuccess;
  const dim3 grid((items + kThreads - 1) / kThreads, nrhs);
  const double d0 = -4.0 * delta + kappa;
  if (zprec == 64)
    k_lat_skeleton<double><<<grid, kThreads, 0, st>>>(v, (double*)z, t.nc, t.link_base, t.nlinks, t.junc_base,
                                                      t.njunc, n, t.lpiv, delta, d0, active);
  else
    k_lat_skeleton<float><<<grid, kThreads, 0, st>>>(v, (float*)z, t.nc, t.link_base, t.nlinks, t.junc_base,
                                                     t.njunc, n, t.lpiv, delta, d0, active);
  return cudaGetLastError();
}

cudaError_t launch_lattice_reduce_rhs(const double* f, const double* q, long long ntot, const LatticeDev& t,
                                      double delta, double* fc, int nrhs, int gx, cudaStream_t st) {
  k_lat_reduce_rhs<<<dim3(gx, nrhs), kThreads, 0, st>>>(f, q, ntot, t.nc, t.anb, delta, fc);
  return cudaGetLastError();
}

cudaError_t launch_lattice_arm_rhs(const double* f, const double* u, long long ntot, const LatticeDev& t,
                                   double delta, double* out, double* p, int nrhs, int gx, cudaStream_t st) {
  k_lat_arm_rhs<<<dim3(gx, nrhs), kThreads, 0, st>>>(f, u, ntot, t.nc, t.gcn, delta, out, p);
  return cudaGetLastError();
}

cudaError_t launch_lattice_global_apply(const double* p, double* y, const double* f, long long ntot,
                                        const LatticeDev& t, double delta, double kappa, double* part, int gmax,
                                        int nrhs, int gx, double* rel_out, double* fnorm_out, double rtol,
                                        double* tolabs, cudaStream_t st) {
  k_lat_global<<<dim3(gx, nrhs), kThreads, 0, st>>>(p, y, f, ntot, t.gnbr, delta, kappa, part, gmax, nrhs);
  if (f) return launch_residual_finalize(part, gmax, gx, nrhs, rel_out, fnorm_out, rtol, tolabs, st);
  return cudaGetLastError();
}

}  // namespace fpg
