// GMRES-side kernels: Schur matvec, Arnoldi (MGS), Givens, cycle end, the
// Schur reduction / back substitution of Alg. "fft_dd_solver", and the global
// operator K for the acceptance residual.  All FP64.
//
// Reductions are deterministic: each CTA reduces its share in a fixed tree and
// writes one partial; the consumer sums the partials of a right-hand side in a
// fixed order (one warp), so a result never depends on scheduling.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fpg_dstline.cuh"
#include "fpg_exactsum.cuh"
#include "fpg_internal.cuh"

namespace fpg {

// Arm slots everywhere: 0 = W, 1 = E, 2 = S, 3 = N (offset < 0 when the arm is absent).

namespace {

constexpr int kThreads = 256;

template <typename Tz>
__device__ __forceinline__ double ld(const Tz* p, long long i) {
  return dl::convert<double>(p[i]);  // integer-pipe widening for FP32 z
}

// Value of C's line that faces arm `a`, position q (0..n-1).
template <typename Tz>
__device__ __forceinline__ double c_line(const Tz* z, int n, int a, int q) {
  switch (a) {
    case 0: return ld(z, (long long)q * n);                 // x = h column
    case 1: return ld(z, (long long)q * n + n - 1);         // x = 1 - h column
    case 2: return ld(z, q);                                // y = h row
    default: return ld(z, (long long)(n - 1) * n + q);      // y = 1 - h row
  }
}

// ---------------------------------------------------------------------------
// a2, reduced form: corr[r][a][i] = sum_j (T(|i-j|) - H(i+j)) line_a[j], i.e.
// delta^2 Q diag(g_k) Q^T applied to C's line next to arm a (the exact interface
// response R_ca A_a^{-1} R_ac restricted to that line; ctab = T[2n+2] then H[2n]).
template <typename Tz>
__global__ void __launch_bounds__(256)
k_schur_lines(const Tz* __restrict__ z, long long zstride, int n, const double* __restrict__ ctab,
              const int* __restrict__ arms, int narms, double* __restrict__ corr,
              const int* __restrict__ active) {
  // CTA: 32 outputs i (threadIdx.x) x 8 column groups (threadIdx.y), each
  // thread one contiguous eighth of the j range (eight short independent FMA
  // chains instead of one long one); the group partials are summed in group
  // order.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* line = reinterpret_cast<double*>(smem_raw);
  double* c = line + n;
  double* hk = c + 2 * n + 2;
  double* part = hk + 2 * n;  // [8][32]
  const int r = blockIdx.y / narms;
  const int a = arms[blockIdx.y % narms];
  if (active != nullptr && !active[r]) return;
  const Tz* zr = z + (long long)r * zstride;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int q = tid; q < n; q += 256) line[q] = c_line(zr, n, a, q);
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
    double s = part[threadIdx.x];
#pragma unroll
    for (int g = 1; g < 8; ++g) s += part[g * 32 + threadIdx.x];
    corr[((long long)r * 4 + a) * n + i] = s;
  }
}

// a2, stencil part fused with the interface corrections:
// w = A_c z - sum_a corr_a on the lines next to the arms.
template <typename Tz>
__global__ void __launch_bounds__(kThreads)
k_stencil_c(const Tz* __restrict__ z, long long zstride, double* __restrict__ w, long long wstride, int n,
            double delta, double kappa, const double* __restrict__ corr, int armmask,
            const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const Tz* zr = z + (long long)r * zstride;
  double* wr = w + (long long)r * wstride;
  const double* cr = corr + (long long)r * 4 * n;
  const long long nc = (long long)n * n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
    const double zc = ld(zr, idx);
    const double s = stencil_sum(zc, i > 0 ? ld(zr, idx - 1) : 0.0, i < n - 1 ? ld(zr, idx + 1) : 0.0,
                                 j > 0 ? ld(zr, idx - n) : 0.0, j < n - 1 ? ld(zr, idx + n) : 0.0);
    double v = fma(delta, s, kappa * zc);
    if (i == 0 && (armmask & 1)) v -= cr[0 * n + j];
    if (i == n - 1 && (armmask & 2)) v -= cr[1 * n + j];
    if (j == 0 && (armmask & 4)) v -= cr[2 * n + i];
    if (j == n - 1 && (armmask & 8)) v -= cr[3 * n + i];
    wr[idx] = v;
  }
}

// a2, literal form, step 1: every arm buffer gets zero except its interface
// line, which receives delta * (C's facing line)  (= R_ac z).
template <typename Tz>
__global__ void k_literal_inject(const Tz* __restrict__ z, long long zstride, int n, double delta,
                                 double* __restrict__ armbuf, long long rhs_stride, ArmOffsets ao,
                                 const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const Tz* zr = z + (long long)r * zstride;
  const int as = ao.as;
  const long long na = (long long)n * as;
  for (int a = 0; a < 4; ++a) {
    if (ao.off[a] < 0) continue;
    double* ab = armbuf + (long long)r * rhs_stride + ao.off[a];
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < na;
         idx += (long long)gridDim.x * blockDim.x) {
      double v = 0.0;
      if (a < 2) {  // W/E: as x n, x fastest
        const int j = (int)(idx / as), i = (int)(idx - (long long)j * as);
        const int iface = (a == 0) ? as - 1 : 0;
        if (i == iface) v = delta * c_line(zr, n, a, j);
      } else {      // S/N: n x as
        const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
        const int iface = (a == 2) ? as - 1 : 0;
        if (j == iface) v = delta * c_line(zr, n, a, i);
      }
      ab[idx] = v;
    }
  }
}

// a2, literal form, step 3: corr = delta * (arm solution on its interface line) (= R_ca A_a^{-1} R_ac z).
__global__ void k_literal_extract(const double* __restrict__ armsol, long long rhs_stride, ArmOffsets ao,
                                  int n, double delta, double* __restrict__ corr,
                                  const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  for (int a = 0; a < 4; ++a) {
    if (ao.off[a] < 0) continue;
    const double* s = armsol + (long long)r * rhs_stride + ao.off[a];
    const int as = ao.as;
    double v;
    if (a == 0) v = s[(long long)q * as + as - 1];
    else if (a == 1) v = s[(long long)q * as];
    else if (a == 2) v = s[(long long)(as - 1) * n + q];
    else v = s[q];
    corr[((long long)r * 4 + a) * n + q] = delta * v;
  }
}

// ---------------------------------------------------------------------------
// a3: modified Gram-Schmidt, one launch per step k of Arnoldi step j.
// Step k (0 <= k <= j+1): fold the previous projection (k >= 1: h_{k-1} from the
// partials of step k-1, w -= h_{k-1} v_{k-1}), then accumulate the partial of
// <w, v_k> (k <= j) or of ||w||^2 (k = j+1).
__global__ void __launch_bounds__(kThreads)
k_mgs_step(const double* __restrict__ V, long long vstride /* per basis vector: nrhs*len */,
           double* __restrict__ w, long long len, int k, int j, int nrhs, double* __restrict__ part,
           int gmax, double* __restrict__ H, int hcol_stride, int hrhs_stride,
           const int* __restrict__ active) {
  __shared__ double red[32];
  __shared__ double hprev_s;
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  double hprev = 0.0;
  if (k >= 1) {
    if (threadIdx.x < 32) {
      const double s = warp_sum_partials(part + ((long long)((k - 1) & 1) * nrhs + r) * gmax, gridDim.x);
      if (threadIdx.x == 0) hprev_s = s;
    }
    __syncthreads();
    hprev = hprev_s;
    if (blockIdx.x == 0 && threadIdx.x == 0 && H != nullptr)
      H[(long long)r * hrhs_stride + (long long)j * hcol_stride + (k - 1)] = hprev;
  }
  double* wr = w + (long long)r * len;
  const double* vp = (k >= 1) ? V + (long long)(k - 1) * vstride + (long long)r * len : nullptr;
  const double* vk = (k <= j) ? V + (long long)k * vstride + (long long)r * len : nullptr;
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    double wv = wr[idx];
    if (vp) {
      wv = fma(-hprev, vp[idx], wv);
      wr[idx] = wv;
    }
    acc = vk ? fma(wv, vk[idx], acc) : fma(wv, wv, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[((long long)(k & 1) * nrhs + r) * gmax + blockIdx.x] = acc;
}

// a3 tail: h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j} (written to vout).
__global__ void __launch_bounds__(kThreads)
k_mgs_normalize(const double* __restrict__ w, double* __restrict__ vout, long long len, int j, int nrhs,
                const double* __restrict__ part, int gmax, double* __restrict__ H, int hcol_stride,
                int hrhs_stride, const int* __restrict__ active) {
  __shared__ double hn_s;
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  if (threadIdx.x < 32) {
    const double s = warp_sum_partials(part + ((long long)((j + 1) & 1) * nrhs + r) * gmax, gridDim.x);
    if (threadIdx.x == 0) hn_s = sqrt(s);
  }
  __syncthreads();
  const double hn = hn_s;
  if (blockIdx.x == 0 && threadIdx.x == 0 && H != nullptr)
    H[(long long)r * hrhs_stride + (long long)j * hcol_stride + (j + 1)] = hn;
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  const double* wr = w + (long long)r * len;
  double* vr = vout + (long long)r * len;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x)
    vr[idx] = wr[idx] * inv;
}

// ---------------------------------------------------------------------------
// a3 + a4 in one launch: one thread-block cluster per right-hand side runs the
// whole modified Gram-Schmidt chain of Arnoldi step j.  Each CTA owns a slice
// of the vector; the dot product of every MGS step is reduced inside the CTA,
// its per-CTA partials are exchanged through distributed shared memory after a
// cluster barrier, and every CTA sums them in the same rank order (so all CTAs
// hold the identical h).  The tail normalises v_{j+1} and, in rank 0, applies
// the Givens step of column j (same arithmetic as k_givens).
__global__ void __launch_bounds__(kThreads)
k_arnoldi_cluster(const double* __restrict__ V, long long vstride, double* __restrict__ w, double* __restrict__ vout,
                  long long len, int j, double* __restrict__ H, int hcol_stride, int hrhs_stride,
                  double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g, double* __restrict__ res,
                  int m, const double* __restrict__ tolabs, int* __restrict__ active, int* __restrict__ kcyc,
                  int* __restrict__ iters, int max_iters, int do_givens) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int csz = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int r = blockIdx.x / csz;
  __shared__ double red[32];
  __shared__ double part[2];
  __shared__ double hval;
  if (active != nullptr && !active[r]) return;  // uniform over the cluster
  const long long chunk = (len + csz - 1) / csz;
  const long long lo = (long long)rank * chunk;
  const long long hi = lo + chunk < len ? lo + chunk : len;
  double* wr = w + (long long)r * len;
  double hprev = 0.0;
  for (int k = 0; k <= j + 1; ++k) {
    const double* vp = (k >= 1) ? V + (long long)(k - 1) * vstride + (long long)r * len : nullptr;
    const double* vk = (k <= j) ? V + (long long)k * vstride + (long long)r * len : nullptr;
    double acc = 0.0;
    for (long long idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
      double wv = wr[idx];
      if (vp) {
        wv = fma(-hprev, vp[idx], wv);
        wr[idx] = wv;
      }
      acc = vk ? fma(wv, vk[idx], acc) : fma(wv, wv, acc);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[k & 1] = acc;
    cl.sync();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int q = 0; q < csz; ++q) sum += *cl.map_shared_rank(&part[k & 1], q);
      hval = sum;
    }
    __syncthreads();
    hprev = hval;
    if (rank == 0 && threadIdx.x == 0 && k <= j) H[(long long)r * hrhs_stride + (long long)j * hcol_stride + k] = hprev;
  }
  const double hn = sqrt(hprev);
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  double* vr = vout + (long long)r * len;
  for (long long idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) vr[idx] = wr[idx] * inv;
  if (rank == 0 && threadIdx.x == 0) {
    double* h = H + (long long)r * hrhs_stride + (long long)j * hcol_stride;
    h[j + 1] = hn;
    if (do_givens) {
      double* c = cs + (long long)r * m;
      double* s = sn + (long long)r * m;
      double* gr = g + (long long)r * (m + 1);
      for (int i = 0; i < j; ++i) {
        const double a = h[i], b = h[i + 1];
        h[i] = c[i] * a + s[i] * b;
        h[i + 1] = -s[i] * a + c[i] * b;
      }
      const double a = h[j], b = h[j + 1];
      const double rr = hypot(a, b);
      double cc = 1.0, ss = 0.0;
      if (rr != 0.0) {
        cc = a / rr;
        ss = b / rr;
      }
      c[j] = cc;
      s[j] = ss;
      h[j] = rr;
      h[j + 1] = 0.0;
      gr[j + 1] = -ss * gr[j];
      gr[j] = cc * gr[j];
      const double rj = fabs(gr[j + 1]);
      res[r] = rj;
      kcyc[r] = j + 1;
      iters[r] += 1;
      if (rj <= tolabs[r] || b == 0.0 || iters[r] >= max_iters) active[r] = 0;
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// Register-resident form of the fused Arnoldi step, for slices of up to
// 16 * 512 elements per CTA (blockDim.x <= kRegMaxThreads, chosen by the host).
// Each thread keeps its EPT elements of w in registers for the whole MGS chain;
// basis vector v_{k+1} is loaded while step k's reduction is in flight, so every
// basis vector is read once, its load latency is hidden, and w is never written
// back.  With z != nullptr the kernel first forms w = A_c z - sum_a corr_a (the
// Schur matvec's stencil, a2) straight into those registers.
//
// Reduction of one MGS step: an exact fixed-point sum (fpg_exactsum.cuh) on the
// integer pipes.  Each warp sums its lanes' partials, warp 0 sums the warps' tuples
// and pushes the CTA's tuple into slot [rank] of every CTA of the cluster with
// st.async (completing on that CTA's mbarrier for the step's parity), then sums the
// csz tuples it received.  Every CTA ends with the same bits; the FP64 pipe, which
// bounds the step, only runs the dot products and updates.  Slot and mbarrier k & 1
// are used again at step k + 2, which no CTA can reach before every CTA has read
// step k's slots (each needs every CTA's step k + 1 tuple first).
constexpr int kRegMaxThreads = 512;
// Tries of each exchange wait.  The exchange cannot give up early and continue
// (the mbarrier phases would fall out of step and late tuples could land in a CTA
// that has left), so the limit only catches a cluster whose CTAs stopped: long
// enough never to fire otherwise.
constexpr int kExchangeTries = 1 << 22;

struct ClusterReduce {
  int4* wtup;                // [16] per-warp tuples
  int4 (*slots)[16];         // [2][16] the cluster's CTA tuples, by step parity
  unsigned long long* mbar;  // [2]
  double* hval;
  int* ok;                   // 0 once an exchange wait gave up
};

__device__ __forceinline__ double cluster_reduce(double acc, int k, const ClusterReduce& R, int csz, int rank) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int4 wt = xs::warp_sum_exact(acc);
  if (lane == 0) R.wtup[wid] = wt;
  __syncthreads();
  if (wid == 0) {
    const int nw = (int)(blockDim.x >> 5);
    const int4 ct = xs::warp_sum_tuples(lane < nw ? R.wtup[lane] : make_int4(0, 0, 0, 0), lane < nw);
    const int b = k & 1;
    if (lane == 0) xs::mbar_expect(&R.mbar[b], (unsigned)(16 * csz));
    __syncwarp();
    if (lane < csz)
      xs::st_async_tuple(xs::cluster_addr(xs::smem_u32(&R.slots[b][rank]), lane), ct,
                         xs::cluster_addr(xs::smem_u32(&R.mbar[b]), lane));
    const bool got = xs::mbar_wait_cluster(&R.mbar[b], (unsigned)((k >> 1) & 1), kExchangeTries);
    const int4 tt = xs::warp_sum_tuples(lane < csz ? R.slots[b][lane] : make_int4(0, 0, 0, 0), lane < csz);
    if (lane == 0) {
      *R.hval = xs::tuple_to_double(tt);
      if (!got) *R.ok = 0;
    }
  }
  __syncthreads();
  return *R.hval;
}

// Largest CTA of the register kernel at EPT elements per thread (keeps w, v_k
// and the prefetched v_{k+1} in registers without spilling).
__host__ __device__ constexpr int reg_max_threads(int ept) { return ept >= 16 ? 256 : kRegMaxThreads; }

template <typename Tz, int EPT>
__global__ void __launch_bounds__(reg_max_threads(EPT), EPT >= 16 ? 2 : 1)
k_arnoldi_cluster_reg(const double* __restrict__ V, long long vstride, const double* __restrict__ w,
                      const Tz* __restrict__ z, const double* __restrict__ corr, int n, double delta, double kappa,
                      int armmask, double* __restrict__ vout, long long len, int j, double* __restrict__ H,
                      int hcol_stride, int hrhs_stride, double* __restrict__ cs, double* __restrict__ sn,
                      double* __restrict__ g, double* __restrict__ res, int m, const double* __restrict__ tolabs,
                      int* __restrict__ active, int* __restrict__ kcyc, int* __restrict__ iters, int max_iters,
                      int do_givens, int* __restrict__ err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int csz = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int r = blockIdx.x / csz;
  __shared__ int4 wtup[kRegMaxThreads / 32];
  __shared__ int4 slots[2][16];
  __shared__ unsigned long long mbar[2];
  __shared__ double hval;
  __shared__ int ok;
  const ClusterReduce R{wtup, slots, mbar, &hval, &ok};
  if (active != nullptr && !active[r]) return;  // uniform over the cluster
  if (threadIdx.x == 0) {
    xs::mbar_init_cluster(&mbar[0]);
    xs::mbar_init_cluster(&mbar[1]);
    ok = 1;
  }
  // Every CTA's mbarriers are initialised before any tuple can reach them: the
  // wait half of this barrier follows the loads below.
  xs::cluster_arrive_release();
  // slice of this CTA: [lo, hi); thread elements lo + tid + e * nb, e < nval
  const int chunk = (int)((len + csz - 1) / csz);
  const int lo = rank * chunk;
  const int hi = (int)(lo + chunk < len ? lo + chunk : len);
  const int nb = blockDim.x, t0 = lo + threadIdx.x;
  const int nval = t0 < hi ? (hi - t0 + nb - 1) / nb : 0;  // valid elements of this thread (<= EPT)
  const long long base = (long long)r * len;
  const double* vt = V + base + t0;  // this thread's first element of v_0
  double wv[EPT], vc[EPT], vn[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) vc[e] = e < nval ? vt[e * nb] : 0.0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int idx = t0 + e * nb;
    double x = 0.0;
    if (e < nval) {
      if (z == nullptr) {
        x = w[base + idx];
      } else {
        const Tz* zr = z + base;
        const double* cr = corr + (long long)r * 4 * n;
        const int jj = idx / n, ii = idx - jj * n;
        const double zc = ld(zr, idx);
        const double sacc = stencil_sum(zc, ii > 0 ? ld(zr, idx - 1) : 0.0, ii < n - 1 ? ld(zr, idx + 1) : 0.0,
                                        jj > 0 ? ld(zr, idx - n) : 0.0, jj < n - 1 ? ld(zr, idx + n) : 0.0);
        x = fma(delta, sacc, kappa * zc);
        if (ii == 0 && (armmask & 1)) x -= cr[0 * n + jj];
        if (ii == n - 1 && (armmask & 2)) x -= cr[1 * n + jj];
        if (jj == 0 && (armmask & 4)) x -= cr[2 * n + ii];
        if (jj == n - 1 && (armmask & 8)) x -= cr[3 * n + ii];
      }
    }
    wv[e] = x;
  }
  xs::cluster_wait_acquire();
  double* hcol = H + (long long)r * hrhs_stride + (long long)j * hcol_stride;
  int kfail = -1;
  for (int k = 0; k <= j; ++k) {
    if (k < j) {  // prefetch v_{k+1}; consumed after this step's reduction
      const double* vk1 = vt + (long long)(k + 1) * vstride;
#pragma unroll
      for (int e = 0; e < EPT; ++e) vn[e] = e < nval ? vk1[e * nb] : 0.0;
    }
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) acc = fma(wv[e], vc[e], acc);
    const double h = cluster_reduce(acc, k, R, csz, rank);
    if (!ok) {
      kfail = k;
      break;
    }
    if (rank == 0 && threadIdx.x == 0) hcol[k] = h;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      wv[e] = fma(-h, vc[e], wv[e]);
      vc[e] = vn[e];
    }
  }
  double hn = 0.0;
  if (kfail < 0) {
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) acc = fma(wv[e], wv[e], acc);
    hn = sqrt(cluster_reduce(acc, j + 1, R, csz, rank));
    if (!ok) kfail = j + 1;
  }
  if (kfail >= 0) {
    // An exchange wait gave up (a CTA of the cluster stopped): report it, give the
    // tuples of that step one more bounded wait to land, and leave without results.
    if (threadIdx.x == 0 && err != nullptr) *err = 1;
    if (threadIdx.x < 32) xs::mbar_wait_cluster(&mbar[kfail & 1], (unsigned)((kfail >> 1) & 1), kExchangeTries);
    return;
  }
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  double* vr = vout + base + t0;
#pragma unroll
  for (int e = 0; e < EPT; ++e)
    if (e < nval) vr[e * nb] = wv[e] * inv;
  if (rank == 0 && threadIdx.x == 0) {
    double* h = hcol;
    h[j + 1] = hn;
    if (do_givens) {
      double* c = cs + (long long)r * m;
      double* s = sn + (long long)r * m;
      double* gr = g + (long long)r * (m + 1);
      for (int i = 0; i < j; ++i) {
        const double a = h[i], b = h[i + 1];
        h[i] = c[i] * a + s[i] * b;
        h[i + 1] = -s[i] * a + c[i] * b;
      }
      const double a = h[j], b = h[j + 1];
      const double rr = hypot(a, b);
      double cc = 1.0, ss = 0.0;
      if (rr != 0.0) {
        cc = a / rr;
        ss = b / rr;
      }
      c[j] = cc;
      s[j] = ss;
      h[j] = rr;
      h[j + 1] = 0.0;
      gr[j + 1] = -ss * gr[j];
      gr[j] = cc * gr[j];
      const double rj = fabs(gr[j + 1]);
      res[r] = rj;
      kcyc[r] = j + 1;
      iters[r] += 1;
      if (rj <= tolabs[r] || b == 0.0 || iters[r] >= max_iters) active[r] = 0;
    }
  }
  // Each CTA waited for the csz tuples of every step, the last included, so no
  // store is in flight towards a CTA when it exits.
}

// ---------------------------------------------------------------------------
// a4: Givens step on column j, one thread per right-hand side.
__global__ void k_givens(double* __restrict__ H, int hcol_stride, int hrhs_stride, double* __restrict__ cs,
                         double* __restrict__ sn, double* __restrict__ g, double* __restrict__ res, int j,
                         int m, int nrhs, const double* __restrict__ tolabs, int* __restrict__ active,
                         int* __restrict__ kcyc, int* __restrict__ iters, int max_iters) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  if (active != nullptr && !active[r]) return;
  double* h = H + (long long)r * hrhs_stride + (long long)j * hcol_stride;
  double* c = cs + (long long)r * m;
  double* s = sn + (long long)r * m;
  double* gr = g + (long long)r * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = c[i] * a + s[i] * b;
    h[i + 1] = -s[i] * a + c[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  const double rr = hypot(a, b);
  double cc = 1.0, ss = 0.0;
  if (rr != 0.0) {
    cc = a / rr;
    ss = b / rr;
  }
  c[j] = cc;
  s[j] = ss;
  h[j] = rr;
  h[j + 1] = 0.0;
  gr[j + 1] = -ss * gr[j];
  gr[j] = cc * gr[j];
  const double rj = fabs(gr[j + 1]);
  res[r] = rj;
  if (kcyc) kcyc[r] = j + 1;
  if (iters) iters[r] += 1;
  if (active != nullptr && tolabs != nullptr) {
    if (rj <= tolabs[r] || b == 0.0 || (iters && iters[r] >= max_iters)) active[r] = 0;
  }
}

// a5: y = R^{-1} g over the kcyc[r] steps of this cycle (one thread per RHS).
__global__ void __launch_bounds__(32)
k_backsolve(const double* __restrict__ H, int hcol_stride, int hrhs_stride, const double* __restrict__ g,
            double* __restrict__ y, int m, int nrhs, const int* __restrict__ kcyc, int h_in_smem) {
  // One warp per right-hand side.  The triangle is staged in shared memory
  // (one coalesced copy) when it fits; each row's dot product is spread over
  // the lanes and reduced in a fixed butterfly, so the chain of k dependent
  // steps costs one reduction each instead of k sequential loads.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* ys = reinterpret_cast<double*>(smem_raw);  // [m]
  double* hs = ys + m;                                  // [hrhs_stride] when staged
  const int r = blockIdx.x, lane = threadIdx.x;
  if (r >= nrhs) return;
  const int k = kcyc[r];
  const double* hg = H + (long long)r * hrhs_stride;
  const double* h = hg;
  if (h_in_smem) {
    for (int i = lane; i < hrhs_stride; i += 32) hs[i] = hg[i];
    h = hs;
  }
  const double* gr = g + (long long)r * (m + 1);
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    double s = 0.0;
    for (int l = i + 1 + lane; l < k; l += 32) s = fma(h[(long long)l * hcol_stride + i], ys[l], s);
    s = warp_sum(s);
    if (lane == 0) ys[i] = (gr[i] - s) / h[(long long)i * hcol_stride + i];
    __syncwarp();
  }
  double* yr = y + (long long)r * m;
  for (int i = lane; i < k; i += 32) yr[i] = ys[i];
}

// a5: u += Z y (k = kcyc[r] columns).
template <typename Tz>
__global__ void __launch_bounds__(kThreads)
k_update_u(double* __restrict__ u, const Tz* __restrict__ Z, long long zvstride, long long len,
           const double* __restrict__ y, int m, const int* __restrict__ kcyc) {
  const int r = blockIdx.y;
  const int k = kcyc[r];
  if (k == 0) return;
  const double* yr = y + (long long)r * m;
  double* ur = u + (long long)r * len;
  const Tz* Zr = Z + (long long)r * len;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    double s = ur[idx];
    for (int i = 0; i < k; ++i) s = fma(yr[i], ld(Zr, (long long)i * zvstride + idx), s);
    ur[idx] = s;
  }
}

// Restart, part 1: rvec = fc - w (w = L_c u); partials of ||rvec||^2.
__global__ void __launch_bounds__(kThreads)
k_residual_partials(const double* __restrict__ fc, const double* __restrict__ w, double* __restrict__ rvec,
                    long long len, int nrhs, double* __restrict__ part, int gmax,
                    const int* __restrict__ done) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  if (done != nullptr && done[r]) return;
  const double* f = fc + (long long)r * len;
  const double* wr = w + (long long)r * len;
  double* rv = rvec + (long long)r * len;
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    const double v = f[idx] - wr[idx];
    rv[idx] = v;
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[(long long)r * gmax + blockIdx.x] = acc;
}

// Restart, part 2: beta = ||rvec||; converged -> done; else v_0 = rvec / beta,
// g = beta e_1, active = 1, kcyc = 0.
__global__ void __launch_bounds__(kThreads)
k_restart(double* __restrict__ v0, long long len, int nrhs, const double* __restrict__ part, int gmax,
          double* __restrict__ g, int m, const double* __restrict__ tolabs, double* __restrict__ rnorm,
          int* __restrict__ done, int* __restrict__ active, int* __restrict__ kcyc,
          const int* __restrict__ iters, int max_iters) {
  __shared__ double beta_s;
  const int r = blockIdx.y;
  if (done[r]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      active[r] = 0;
      kcyc[r] = 0;
    }
    return;
  }
  if (threadIdx.x < 32) {
    const double s = warp_sum_partials(part + (long long)r * gmax, gridDim.x);
    if (threadIdx.x == 0) beta_s = sqrt(s);
  }
  __syncthreads();
  const double beta = beta_s;
  const bool conv = beta <= tolabs[r];
  const bool out_of_steps = iters[r] >= max_iters;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    rnorm[r] = beta;
    kcyc[r] = 0;
    if (conv || out_of_steps) {
      done[r] = 1;
      active[r] = 0;
    } else {
      active[r] = 1;
      double* gr = g + (long long)r * (m + 1);
      gr[0] = beta;
      for (int i = 1; i <= m; ++i) gr[i] = 0.0;
    }
  }
  if (conv || out_of_steps) return;
  const double inv = 1.0 / beta;
  double* vr = v0 + (long long)r * len;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x)
    vr[idx] *= inv;
}

// ---------------------------------------------------------------------------
// a6: Alg. 1 step 3, f'_c = f_c - sum_a R_ca q_a, with q_a held in the arm
// blocks of `q` (full vectors).  R_ca picks delta * (arm value on its interface line).
__global__ void __launch_bounds__(kThreads)
k_reduce_rhs(const double* __restrict__ f, const double* __restrict__ q, long long ntot, int n,
             double delta, ArmOffsets ao, double* __restrict__ fc) {
  const int r = blockIdx.y;
  const double* fr = f + (long long)r * ntot;
  const double* qr = q + (long long)r * ntot;
  double* out = fc + (long long)r * n * n;
  const long long nc = (long long)n * n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
    double v = fr[idx];
    const int as = ao.as;
    if (i == 0 && ao.off[0] >= 0) v -= delta * qr[ao.off[0] + (long long)j * as + as - 1];
    if (i == n - 1 && ao.off[1] >= 0) v -= delta * qr[ao.off[1] + (long long)j * as];
    if (j == 0 && ao.off[2] >= 0) v -= delta * qr[ao.off[2] + (long long)(as - 1) * n + i];
    if (j == n - 1 && ao.off[3] >= 0) v -= delta * qr[ao.off[3] + i];
    out[idx] = v;
  }
}

// a6: Alg. 1 step 5, f'_a = f_a - R_ac p_c for every arm (into `out`, full vectors),
// and the centre block of `p` receives u.
__global__ void __launch_bounds__(kThreads)
k_arm_rhs(const double* __restrict__ f, const double* __restrict__ u, long long ntot, int n, double delta,
          ArmOffsets ao, double* __restrict__ out, double* __restrict__ p) {
  const int r = blockIdx.y;
  const double* fr = f + (long long)r * ntot;
  const double* ur = u + (long long)r * n * n;
  double* o = out + (long long)r * ntot;
  double* pr = p + (long long)r * ntot;
  const long long nc = (long long)n * n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ntot;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nc) {
      pr[idx] = ur[idx];
      continue;
    }
    double v = fr[idx];
    const int as = ao.as;
    for (int a = 0; a < 4; ++a) {
      const long long off = ao.off[a];
      if (off < 0 || idx < off || idx >= off + (long long)n * as) continue;
      const long long li = idx - off;
      if (a < 2) {
        const int j = (int)(li / as), i = (int)(li - (long long)j * as);
        if (a == 0 && i == as - 1) v -= delta * ur[(long long)j * n];
        if (a == 1 && i == 0) v -= delta * ur[(long long)j * n + n - 1];
      } else {
        const int j = (int)(li / n), i = (int)(li - (long long)j * n);
        if (a == 2 && j == as - 1) v -= delta * ur[i];
        if (a == 3 && j == 0) v -= delta * ur[(long long)(n - 1) * n + i];
      }
    }
    o[idx] = v;
  }
}

// Ghost value beyond an arm's own edge (the arm seen alone, its interface line
// treated as Dirichlet): 0 on the vertex-centred grid; on the cell-centred grid
// (bc = 1) 0 across the interface, xc across a side (Neumann face), -xc across
// the far end (Dirichlet face).  side: 0 = interface, 1 = side, 2 = far end.
__device__ __forceinline__ double arm_ghost(int bc, int side, double xc) {
  if (bc == 0 || side == 0) return 0.0;
  return side == 1 ? xc : -xc;
}

// a6 refinement: out_a = rhs_a - A_a x_a on every arm block (A_a: the arm's own
// 5-point operator, its interface line treated as Dirichlet), full-vector layout.
__global__ void __launch_bounds__(kThreads)
k_arm_residual(const double* __restrict__ rhs, const double* __restrict__ x, double* __restrict__ out,
               long long ntot, int n, double delta, double kappa, ArmOffsets ao) {
  const int r = blockIdx.y;
  const int as = ao.as, bc = ao.bc;
  const long long na = (long long)n * as;
  for (int a = 0; a < 4; ++a) {
    const long long off = ao.off[a];
    if (off < 0) continue;
    const int nx = a < 2 ? as : n, ny = a < 2 ? n : as;
    // which edge lies beyond i = -1, i = nx, j = -1, j = ny
    const int eL = a == 0 ? 2 : (a == 1 ? 0 : 1), eR = a == 0 ? 0 : (a == 1 ? 2 : 1);
    const int eD = a == 2 ? 2 : (a == 3 ? 0 : 1), eU = a == 2 ? 0 : (a == 3 ? 2 : 1);
    const double* xr = x + (long long)r * ntot + off;
    const double* fr = rhs + (long long)r * ntot + off;
    double* o = out + (long long)r * ntot + off;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < na;
         idx += (long long)gridDim.x * blockDim.x) {
      const int j = (int)(idx / nx), i = (int)(idx - (long long)j * nx);
      const double xc = xr[idx];
      const double s = stencil_sum(xc, i > 0 ? xr[idx - 1] : arm_ghost(bc, eL, xc),
                                   i < nx - 1 ? xr[idx + 1] : arm_ghost(bc, eR, xc),
                                   j > 0 ? xr[idx - nx] : arm_ghost(bc, eD, xc),
                                   j < ny - 1 ? xr[idx + nx] : arm_ghost(bc, eU, xc));
      o[idx] = fr[idx] - fma(delta, s, kappa * xc);
    }
  }
}

// x_a += e_a on every arm block.
__global__ void __launch_bounds__(kThreads)
k_arm_add(double* __restrict__ x, const double* __restrict__ e, long long ntot, int n, ArmOffsets ao) {
  const int r = blockIdx.y;
  const long long na = (long long)n * ao.as;
  for (int a = 0; a < 4; ++a) {
    const long long off = ao.off[a];
    if (off < 0) continue;
    double* xr = x + (long long)r * ntot + off;
    const double* er = e + (long long)r * ntot + off;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < na;
         idx += (long long)gridDim.x * blockDim.x)
      xr[idx] += er[idx];
  }
}

// ---------------------------------------------------------------------------
// Global operator K (a7): value of the neighbour (di, dj) of local node (i, j)
// of block `blk` (0 = C, 1..4 = W, E, S, N) whose own value is pc.  Beyond the
// domain's edge: zero on the vertex-centred grid; on the cell-centred grid
// (bc = 1) pc across an arm's side (Neumann face) and -pc across its far end
// (Dirichlet face).
__device__ __forceinline__ double nb_value(const double* pr, int n, const ArmOffsets& ao, int blk, int i,
                                           int j, int di, int dj, double pc) {
  const int ni = i + di, nj = j + dj;
  const int as = ao.as;
  if (blk == 0) {
    if (ni >= 0 && ni < n && nj >= 0 && nj < n) return pr[(long long)nj * n + ni];
    if (ni < 0) return ao.off[0] >= 0 ? pr[ao.off[0] + (long long)nj * as + as - 1] : 0.0;
    if (ni >= n) return ao.off[1] >= 0 ? pr[ao.off[1] + (long long)nj * as] : 0.0;
    if (nj < 0) return ao.off[2] >= 0 ? pr[ao.off[2] + (long long)(as - 1) * n + ni] : 0.0;
    return ao.off[3] >= 0 ? pr[ao.off[3] + ni] : 0.0;
  }
  const int a = blk - 1;
  const long long off = ao.off[a];
  if (a < 2) {  // as x n
    if (ni >= 0 && ni < as && nj >= 0 && nj < n) return pr[off + (long long)nj * as + ni];
    if (a == 0 && ni == as) return pr[(long long)nj * n];             // W -> C column 0
    if (a == 1 && ni == -1) return pr[(long long)nj * n + n - 1];     // E -> C column n-1
    if (ao.bc == 0) return 0.0;
    return (nj < 0 || nj >= n) ? pc : -pc;                            // side : far end
  }
  if (ni >= 0 && ni < n && nj >= 0 && nj < as) return pr[off + (long long)nj * n + ni];
  if (a == 2 && nj == as) return pr[ni];                              // S -> C row 0
  if (a == 3 && nj == -1) return pr[(long long)(n - 1) * n + ni];     // N -> C row n-1
  if (ao.bc == 0) return 0.0;
  return (ni < 0 || ni >= n) ? pc : -pc;                              // side : far end
}

__device__ __forceinline__ void locate(long long idx, int n, const ArmOffsets& ao, int* blk, int* i, int* j) {
  const long long nc = (long long)n * n;
  if (idx < nc) {
    *blk = 0;
    *j = (int)(idx / n);
    *i = (int)(idx - (long long)(*j) * n);
    return;
  }
  for (int a = 0; a < 4; ++a) {
    const long long off = ao.off[a];
    if (off < 0 || idx < off || idx >= off + (long long)n * ao.as) continue;
    const long long li = idx - off;
    *blk = a + 1;
    const int nx = (a < 2) ? ao.as : n;
    *j = (int)(li / nx);
    *i = (int)(li - (long long)(*j) * nx);
    return;
  }
  *blk = -1;
  *i = *j = 0;
}

// y = K p; with f != nullptr also accumulates partials of ||f - K p||^2 and ||f||^2.
__global__ void __launch_bounds__(kThreads)
k_global_apply(const double* __restrict__ p, double* __restrict__ y, const double* __restrict__ f,
               long long ntot, int n, double delta, double kappa, ArmOffsets ao, double* __restrict__ part,
               int gmax, int nrhs) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  const double* pr = p + (long long)r * ntot;
  double rr = 0.0, ff = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ntot;
       idx += (long long)gridDim.x * blockDim.x) {
    int blk, i, j;
    locate(idx, n, ao, &blk, &i, &j);
    const double pc = pr[idx];
    const double s = stencil_sum(pc, nb_value(pr, n, ao, blk, i, j, -1, 0, pc), nb_value(pr, n, ao, blk, i, j, 1, 0, pc),
                                 nb_value(pr, n, ao, blk, i, j, 0, -1, pc), nb_value(pr, n, ao, blk, i, j, 0, 1, pc));
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

// out[r] = sqrt(sum rr) / sqrt(sum ff) (relative residual); fnorm_out[r] = sqrt(sum ff).
__global__ void k_residual_finalize(const double* __restrict__ part, int gmax, int cnt, int nrhs,
                                    double* __restrict__ out, double* __restrict__ fnorm_out,
                                    double rtol, double* __restrict__ tolabs) {
  const int r = blockIdx.x;
  if (threadIdx.x >= 32) return;
  const double rr = warp_sum_partials(part + ((long long)0 * nrhs + r) * gmax, cnt);
  const double ff = warp_sum_partials(part + ((long long)1 * nrhs + r) * gmax, cnt);
  if (threadIdx.x == 0) {
    const double fn = sqrt(ff);
    if (out) out[r] = fn > 0.0 ? sqrt(rr) / fn : sqrt(rr);
    if (fnorm_out) fnorm_out[r] = fn;
    if (tolabs) tolabs[r] = rtol * fn;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Comparison preconditioners of Sec. 3.2 (P = I and the Jacobi P = D_2).
// Jacobi: z = v / diag(L_c) with diag(L_c) = -4 delta + kappa on C, minus, on the
// line next to arm a, the diagonal of delta^2 Q diag(g) Q^T, which is T(0) - H(2q)
// at position q of that line (the Toeplitz-plus-Hankel form of the interface table).
template <typename To>
__global__ void __launch_bounds__(kThreads)
k_precond_simple(const double* __restrict__ v, To* __restrict__ z, long long len, int n, double delta, double kappa,
                 const double* __restrict__ ctab, int armmask, int jacobi, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const double* vr = v + (long long)r * len;
  To* zr = z + (long long)r * len;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    double x = vr[idx];
    if (jacobi) {
      const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
      const double* hk = ctab + 2 * n + 2;
      double d = -4.0 * delta + kappa;
      if (i == 0 && (armmask & 1)) d -= ctab[0] - hk[2 * j];
      if (i == n - 1 && (armmask & 2)) d -= ctab[0] - hk[2 * j];
      if (j == 0 && (armmask & 4)) d -= ctab[0] - hk[2 * i];
      if (j == n - 1 && (armmask & 8)) d -= ctab[0] - hk[2 * i];
      x /= d;
    }
    zr[idx] = (To)x;
  }
}

// Acceptance check (P8 reading): a right-hand side whose global residual is above
// rtol after back substitution goes back into the iteration with its Schur
// tolerance scaled by `factor`; its iterate u is kept.  Flags how many resume.

// Global iterative refinement (acceptance, a7): r = f - K p for the right-hand
// sides whose global relative residual is above rtol, 0 for the others (those
// then converge at once and their correction is exactly zero).  On entry r
// holds K p.
__global__ void __launch_bounds__(kThreads)
k_refine_rhs(const double* __restrict__ f, double* __restrict__ r, const double* __restrict__ gres, double rtol,
             long long ntot, int* __restrict__ resume_count) {
  const int rr = blockIdx.y;
  const bool refine = gres[rr] > rtol;
  if (refine && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(resume_count, 1);
  const double* fr = f + (long long)rr * ntot;
  double* xr = r + (long long)rr * ntot;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += (long long)gridDim.x * blockDim.x)
    xr[i] = refine ? fr[i] - xr[i] : 0.0;
}

__global__ void __launch_bounds__(kThreads)
k_add_vec(double* __restrict__ p, const double* __restrict__ q, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    p[i] += q[i];
}

__global__ void k_refine_tol(double* __restrict__ tolabs, const double* __restrict__ fnorm0, double scale, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) tolabs[r] = scale * fnorm0[r];
}

// ---------------------------------------------------------------------------
// Launchers (library-internal).
// a2, reduced form as a matrix product: corr[r][a][i] = sum_j G(j, i) line_a[j] with
// the interface matrix G(i, j) = T(|i-j|) - H(i+j) of the table above stored whole
// (n x n, symmetric, built once per domain).  One CTA takes 16 outputs i of every arm
// line of one right-hand side, the j range split over 16 groups of threads: each
// element of G (read coalesced from L2) feeds one FMA per arm, where the table form
// spends a subtraction and an FMA per arm and output.  Group partials are summed in
// group order (deterministic).
constexpr int kGTile = 16, kGGroups = 16;

template <typename Tz>
__global__ void __launch_bounds__(kGTile * kGGroups)
k_schur_lines_g(const Tz* __restrict__ z, long long zstride, int n, const double* __restrict__ G,
                const int* __restrict__ arms, int narms, double* __restrict__ corr, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* line = reinterpret_cast<double*>(smem_raw);  // [narms][n]
  double* part = line + 4 * n;                         // [kGGroups][4][kGTile]
  const int r = blockIdx.y;
  if (active != nullptr && !active[r]) return;
  const Tz* zr = z + (long long)r * zstride;
  for (int q = threadIdx.x; q < narms * n; q += kGTile * kGGroups) {
    const int a = q / n;
    line[q] = c_line(zr, n, arms[a], q - a * n);
  }
  __syncthreads();
  const int tx = threadIdx.x % kGTile, ty = threadIdx.x / kGTile;
  const int i = blockIdx.x * kGTile + tx;
  const int per = (n + kGGroups - 1) / kGGroups;
  const int j0 = ty * per, j1 = min(n, j0 + per);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    // eight elements of G in flight before their FMAs (the loop is bound by L2 latency)
    constexpr int U = 8;
    const double* gp = G + (long long)j0 * n + i;
    int j = j0;
    for (; j + U <= j1; j += U, gp += (long long)U * n) {
      double g[U];
#pragma unroll
      for (int u = 0; u < U; ++u) g[u] = gp[(long long)u * n];
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (a < narms) acc[a] = fma(g[u], line[a * n + j + u], acc[a]);
      }
    }
    for (; j < j1; ++j, gp += n) {
      const double g = *gp;
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (a < narms) acc[a] = fma(g, line[a * n + j], acc[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) part[(ty * 4 + a) * kGTile + tx] = acc[a];
  __syncthreads();
  if (threadIdx.x < 4 * kGTile) {
    const int a = threadIdx.x / kGTile, t2 = threadIdx.x % kGTile;
    const int i2 = blockIdx.x * kGTile + t2;
    if (a < narms && i2 < n) {
      double sum = part[a * kGTile + t2];
      for (int g = 1; g < kGGroups; ++g) sum += part[(g * 4 + a) * kGTile + t2];
      corr[((long long)r * 4 + arms[a]) * n + i2] = sum;
    }
  }
}

cudaError_t launch_schur_gmat(const void* z, int zprec, long long zstride, int n, const double* G, const int* arms_dev,
                              int narms, double* corr, const int* active, int nrhs, cudaStream_t st) {
  if (narms < 1 || narms > 4) return cudaErrorInvalidValue;
  dim3 grid((n + kGTile - 1) / kGTile, nrhs);
  const size_t smem = sizeof(double) * (4 * (size_t)n + kGGroups * 4 * kGTile);
  static PerDeviceOnce attr_set;
  if (auto once = attr_set.first()) {
    cudaFuncSetAttribute(k_schur_lines_g<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_schur_lines_g<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  if (zprec == 64)
    k_schur_lines_g<double><<<grid, kGTile * kGGroups, smem, st>>>((const double*)z, zstride, n, G, arms_dev, narms,
                                                                   corr, active);
  else
    k_schur_lines_g<float><<<grid, kGTile * kGGroups, smem, st>>>((const float*)z, zstride, n, G, arms_dev, narms,
                                                                  corr, active);
  return cudaGetLastError();
}

cudaError_t launch_schur_reduced(const void* z, int zprec, long long zstride, int n, const double* ctab,
                                 const int* arms_dev, int narms, double* corr, const int* active, int nrhs,
                                 cudaStream_t st) {
  dim3 grid((n + 31) / 32, nrhs * narms);
  const size_t smem = sizeof(double) * (5 * n + 2 + 256);
  static PerDeviceOnce attr_set;
  if (auto once = attr_set.first()) {
    cudaFuncSetAttribute(k_schur_lines<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_schur_lines<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  if (zprec == 64)
    k_schur_lines<double><<<grid, dim3(32, 8), smem, st>>>((const double*)z, zstride, n, ctab, arms_dev, narms,
                                                            corr, active);
  else
    k_schur_lines<float><<<grid, dim3(32, 8), smem, st>>>((const float*)z, zstride, n, ctab, arms_dev, narms,
                                                           corr, active);
  return cudaGetLastError();
}

cudaError_t launch_precond_simple(const double* v, void* z, int zprec, long long len, int n, double delta,
                                  double kappa, const double* ctab, int armmask, int jacobi, const int* active,
                                  int nrhs, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  if (zprec == 64)
    k_precond_simple<double><<<grid, kThreads, 0, st>>>(v, (double*)z, len, n, delta, kappa, ctab, armmask, jacobi,
                                                        active);
  else
    k_precond_simple<float><<<grid, kThreads, 0, st>>>(v, (float*)z, len, n, delta, kappa, ctab, armmask, jacobi,
                                                       active);
  return cudaGetLastError();
}

cudaError_t launch_refine_rhs(const double* f, double* r, const double* gres, double rtol, long long ntot, int nrhs,
                              int* resume_count, int gx, cudaStream_t st) {
  k_refine_rhs<<<dim3(gx, nrhs), kThreads, 0, st>>>(f, r, gres, rtol, ntot, resume_count);
  return cudaGetLastError();
}

cudaError_t launch_add_vec(double* p, const double* q, long long total, cudaStream_t st) {
  const long long blocks = (total + kThreads - 1) / kThreads;
  k_add_vec<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), kThreads, 0, st>>>(p, q, total);
  return cudaGetLastError();
}

cudaError_t launch_refine_tol(double* tolabs, const double* fnorm0, double scale, int nrhs, cudaStream_t st) {
  k_refine_tol<<<(nrhs + 127) / 128, 128, 0, st>>>(tolabs, fnorm0, scale, nrhs);
  return cudaGetLastError();
}


cudaError_t launch_stencil_c(const void* z, int zprec, long long zstride, double* w, long long wstride, int n,
                             double delta, double kappa, const double* corr, int armmask, const int* active,
                             int nrhs, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  if (zprec == 64)
    k_stencil_c<double><<<grid, kThreads, 0, st>>>((const double*)z, zstride, w, wstride, n, delta, kappa, corr,
                                                    armmask, active);
  else
    k_stencil_c<float><<<grid, kThreads, 0, st>>>((const float*)z, zstride, w, wstride, n, delta, kappa, corr,
                                                   armmask, active);
  return cudaGetLastError();
}

cudaError_t launch_literal_inject(const void* z, int zprec, long long zstride, int n, double delta,
                                  double* armbuf, long long rhs_stride, ArmOffsets ao, const int* active,
                                  int nrhs, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  if (zprec == 64)
    k_literal_inject<double><<<grid, kThreads, 0, st>>>((const double*)z, zstride, n, delta, armbuf, rhs_stride,
                                                         ao, active);
  else
    k_literal_inject<float><<<grid, kThreads, 0, st>>>((const float*)z, zstride, n, delta, armbuf, rhs_stride,
                                                        ao, active);
  return cudaGetLastError();
}

cudaError_t launch_literal_extract(const double* armsol, long long rhs_stride, ArmOffsets ao, int n,
                                   double delta, double* corr, const int* active, int nrhs, cudaStream_t st) {
  dim3 grid((n + 127) / 128, nrhs);
  k_literal_extract<<<grid, 128, 0, st>>>(armsol, rhs_stride, ao, n, delta, corr, active);
  return cudaGetLastError();
}

cudaError_t launch_mgs(const double* V, long long vstride, double* w, double* vout, long long len, int j,
                       int nrhs, double* part, int gmax, double* H, int hcol_stride, int hrhs_stride,
                       const int* active, int gx, cudaStream_t st, int* launches) {
  dim3 grid(gx, nrhs);
  for (int k = 0; k <= j + 1; ++k) {
    k_mgs_step<<<grid, kThreads, 0, st>>>(V, vstride, w, len, k, j, nrhs, part, gmax, H, hcol_stride,
                                          hrhs_stride, active);
  }
  k_mgs_normalize<<<grid, kThreads, 0, st>>>(w, vout, len, j, nrhs, part, gmax, H, hcol_stride, hrhs_stride,
                                             active);
  if (launches) *launches += j + 3;
  return cudaGetLastError();
}

// Cluster size for the fused Arnoldi kernel, 0 when the multi-launch MGS is
// the better choice (long vectors: a 16-CTA cluster would leave the GPU idle).
int arnoldi_cluster_size(long long len) {
  if (len > 262144) return 0;
  long long c = (len + 2047) / 2048;
  if (c > 16) c = 16;
  if (c < 1) c = 1;
  return (int)c;
}

cudaError_t launch_arnoldi_cluster(int csz, const double* V, long long vstride, double* w, double* vout,
                                   long long len, int j, int nrhs, double* H, int hcol_stride, int hrhs_stride,
                                   double* cs, double* sn, double* g, double* res, int m, const double* tolabs,
                                   int* active, int* kcyc, int* iters, int max_iters, int do_givens,
                                   cudaStream_t st) {
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_arnoldi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csz * nrhs, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_arnoldi_cluster, V, vstride, w, vout, len, j, H, hcol_stride, hrhs_stride, cs,
                            sn, g, res, m, tolabs, active, kcyc, iters, max_iters, do_givens);
}

// Register-resident fused Arnoldi: returns cudaErrorInvalidValue when the
// slice per CTA is too long for it (the caller then uses k_arnoldi_cluster).
// Elements per thread of the register Arnoldi kernel for a slice of
// ceil(len/csz) elements under a cap of ntcap threads per CTA (0: 256 when the
// slice fits, else 512 -- narrow CTAs with 16 elements each let two domains'
// kernels share an SM); 0 when the slice is too long.
int arnoldi_reg_ept(long long len, int csz, int ntcap) {
  if (ntcap <= 0) {
    const int e = arnoldi_reg_ept(len, csz, 256);
    return e > 0 ? e : arnoldi_reg_ept(len, csz, kRegMaxThreads);
  }
  if (ntcap > kRegMaxThreads) ntcap = kRegMaxThreads;
  const long long chunk = (len + csz - 1) / csz;
  static const int epts[] = {2, 4, 8, 12, 16};
  for (int e : epts) {
    const long long nt = ((chunk + e - 1) / e + 31) / 32 * 32;
    if (nt <= ntcap && nt <= reg_max_threads(e)) return e;
  }
  return 0;
}

// Threads per CTA for a slice of ceil(len/csz) elements at EPT per thread.
int arnoldi_reg_threads(long long len, int csz, int ept) {
  const long long chunk = (len + csz - 1) / csz;
  const long long t = (chunk + ept - 1) / ept;
  return (int)((t + 31) / 32 * 32);
}

template <typename Tz, int EPT>
cudaError_t launch_reg_impl(int csz, const double* V, long long vstride, const double* w, const Tz* z,
                            const double* corr, int n, double delta, double kappa, int armmask, double* vout,
                            long long len, int j, int nrhs, double* H, int hcol_stride, int hrhs_stride, double* cs,
                            double* sn, double* g, double* res, int m, const double* tolabs, int* active, int* kcyc,
                            int* iters, int max_iters, int do_givens, int* err, cudaStream_t st) {
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_arnoldi_cluster_reg<Tz, EPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csz * nrhs, 1, 1);
  cfg.blockDim = dim3(arnoldi_reg_threads(len, csz, EPT), 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_arnoldi_cluster_reg<Tz, EPT>, V, vstride, w, z, corr, n, delta, kappa, armmask,
                            vout, len, j, H, hcol_stride, hrhs_stride, cs, sn, g, res, m, tolabs, active, kcyc,
                            iters, max_iters, do_givens, err);
}

// z == nullptr: w is read from `w`; otherwise w = A_c z - corr is formed in the kernel (zprec 64 or 32).
cudaError_t launch_arnoldi_reg(int csz, int ntcap, const double* V, long long vstride, const double* w,
                               const void* z, int zprec, const double* corr, int n, double delta, double kappa, int armmask,
                               double* vout, long long len, int j, int nrhs, double* H, int hcol_stride,
                               int hrhs_stride, double* cs, double* sn, double* g, double* res, int m,
                               const double* tolabs, int* active, int* kcyc, int* iters, int max_iters, int do_givens,
                               int* err, cudaStream_t st) {
  const int ept = arnoldi_reg_ept(len, csz, ntcap);
#define FPG_REG_CASE(E)                                                                                            \
  if (ept == E) {                                                                                                  \
    if (z != nullptr && zprec == 32)                                                                               \
      return launch_reg_impl<float, E>(csz, V, vstride, w, (const float*)z, corr, n, delta, kappa, armmask, vout,  \
                                       len, j, nrhs, H, hcol_stride, hrhs_stride, cs, sn, g, res, m, tolabs, active, \
                                       kcyc, iters, max_iters, do_givens, err, st);                                \
    return launch_reg_impl<double, E>(csz, V, vstride, w, (const double*)z, corr, n, delta, kappa, armmask, vout,  \
                                      len, j, nrhs, H, hcol_stride, hrhs_stride, cs, sn, g, res, m, tolabs, active, \
                                      kcyc, iters, max_iters, do_givens, err, st);                                 \
  }
  FPG_REG_CASE(2)
  FPG_REG_CASE(4)
  FPG_REG_CASE(8)
  FPG_REG_CASE(12)
  FPG_REG_CASE(16)
#undef FPG_REG_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_givens(double* H, int hcol_stride, int hrhs_stride, double* cs, double* sn, double* g,
                          double* res, int j, int m, int nrhs, const double* tolabs, int* active, int* kcyc,
                          int* iters, int max_iters, cudaStream_t st) {
  k_givens<<<(nrhs + 63) / 64, 64, 0, st>>>(H, hcol_stride, hrhs_stride, cs, sn, g, res, j, m, nrhs, tolabs,
                                            active, kcyc, iters, max_iters);
  return cudaGetLastError();
}

cudaError_t launch_cycle_end(const double* H, int hcol_stride, int hrhs_stride, const double* g, double* y,
                             int m, int nrhs, const int* kcyc, double* u, const void* Z, int zprec,
                             long long zvstride, long long len, int gx, cudaStream_t st) {
  const size_t hbytes = sizeof(double) * (size_t)hrhs_stride;
  const int staged = sizeof(double) * (size_t)m + hbytes <= 48 * 1024 ? 1 : 0;
  k_backsolve<<<nrhs, 32, sizeof(double) * (size_t)m + (staged ? hbytes : 0), st>>>(H, hcol_stride, hrhs_stride, g,
                                                                                   y, m, nrhs, kcyc, staged);
  dim3 grid(gx, nrhs);
  if (zprec == 64)
    k_update_u<double><<<grid, kThreads, 0, st>>>(u, (const double*)Z, zvstride, len, y, m, kcyc);
  else
    k_update_u<float><<<grid, kThreads, 0, st>>>(u, (const float*)Z, zvstride, len, y, m, kcyc);
  return cudaGetLastError();
}

cudaError_t launch_restart(const double* fc, const double* w, double* v0, long long len, int nrhs, double* part,
                           int gmax, double* g, int m, const double* tolabs, double* rnorm, int* done,
                           int* active, int* kcyc, const int* iters, int max_iters, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  k_residual_partials<<<grid, kThreads, 0, st>>>(fc, w, v0, len, nrhs, part, gmax, done);
  k_restart<<<grid, kThreads, 0, st>>>(v0, len, nrhs, part, gmax, g, m, tolabs, rnorm, done, active, kcyc, iters,
                                       max_iters);
  return cudaGetLastError();
}

cudaError_t launch_reduce_rhs(const double* f, const double* q, long long ntot, int n, double delta,
                              ArmOffsets ao, double* fc, int nrhs, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  k_reduce_rhs<<<grid, kThreads, 0, st>>>(f, q, ntot, n, delta, ao, fc);
  return cudaGetLastError();
}

cudaError_t launch_arm_rhs(const double* f, const double* u, long long ntot, int n, double delta, ArmOffsets ao,
                           double* out, double* p, int nrhs, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  k_arm_rhs<<<grid, kThreads, 0, st>>>(f, u, ntot, n, delta, ao, out, p);
  return cudaGetLastError();
}

cudaError_t launch_arm_residual(const double* rhs, const double* x, double* out, long long ntot, int n, double delta,
                                double kappa, ArmOffsets ao, int nrhs, int gx, cudaStream_t st) {
  dim3 grid(gx, nrhs);
  k_arm_residual<<<grid, kThreads, 0, st>>>(rhs, x, out, ntot, n, delta, kappa, ao);
  return cudaGetLastError();
}

cudaError_t launch_arm_add(double* x, const double* e, long long ntot, int n, ArmOffsets ao, int nrhs, int gx,
                           cudaStream_t st) {
  dim3 grid(gx, nrhs);
  k_arm_add<<<grid, kThreads, 0, st>>>(x, e, ntot, n, ao);
  return cudaGetLastError();
}

cudaError_t launch_residual_finalize(const double* part, int gmax, int cnt, int nrhs, double* out, double* fnorm_out,
                                     double rtol, double* tolabs, cudaStream_t st) {
  k_residual_finalize<<<nrhs, 32, 0, st>>>(part, gmax, cnt, nrhs, out, fnorm_out, rtol, tolabs);
  return cudaGetLastError();
}

cudaError_t launch_global_apply(const double* p, double* y, const double* f, long long ntot, int n, double delta,
                                double kappa, ArmOffsets ao, double* part, int gmax, int nrhs, int gx,
                                double* rel_out, double* fnorm_out, double rtol, double* tolabs,
                                cudaStream_t st) {
  dim3 grid(gx, nrhs);
  k_global_apply<<<grid, kThreads, 0, st>>>(p, y, f, ntot, n, delta, kappa, ao, part, gmax, nrhs);
  if (f) k_residual_finalize<<<nrhs, 32, 0, st>>>(part, gmax, gx, nrhs, rel_out, fnorm_out, rtol, tolabs);
  return cudaGetLastError();
}

}  // namespace fpg
