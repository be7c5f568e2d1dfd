// Fused fast solve: z = A^{-1} v for a batch of Dirichlet rectangles in ONE
// pass over HBM (read v once, write z once), one thread-block cluster per block.
//
// The block's ns lines are split into strips of R consecutive lines, one strip
// per CTA of the cluster; the whole block's spectral coefficients stay in the
// cluster's shared memory between the three steps of Sec. 2.1:
//   1. every CTA applies the DST-I to its lines (the shared-memory FFT engine of
//      fpg_dst.cuh, 2Q lines at a time) and keeps the coefficients [R][n];
//   2. the per-mode tridiagonal solves of Eq. "trans_subeq" run across the
//      strips: each CTA evaluates the two Thomas recurrences (y_s = r_s f_s +
//      m_s y_{s-1}, x_s = y_s + m_s x_{s+1}, m_s = -delta r_s) on its own lines
//      with a zero carry, publishes the (chunk result, chunk multiplier) pair of
//      every mode in shared memory, and after a cluster barrier reads the pairs
//      of the other CTAs through distributed shared memory to form its carry;
//   3. every CTA applies the inverse DST-I (x 2/(n+1)) to its lines and stores.
// Same arithmetic as the three-kernel path up to the association of the
// carries.  Blocks too large for one cluster's shared memory (n = 1024 in
// FP32 or FP64) use the three-kernel path instead.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"

namespace fpg {
namespace {

constexpr int kThreads = 256;

template <typename T, typename To, int MAXR>
__global__ void __launch_bounds__(kThreads)
k_fast_solve_fused(const double* __restrict__ in, BatchDesc ib, To* __restrict__ out, BatchDesc ob, LineLayout L,
                   DstPlan pl, const T* __restrict__ rpiv, const T* __restrict__ mneg, int R, int Q,
                   const int* __restrict__ active, int nper_active) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int csz = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;  // uniform over the cluster (same b)
  const int n = pl.n, ns = L.ns;
  const int s0 = min(ns, rank * R);
  const int s1 = min(ns, s0 + R);
  const int nloc = s1 - s0;
  const int lpb = 2 * Q;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* coef = reinterpret_cast<T*>(smem_raw);  // [R][n]
  T* exf = coef + (size_t)R * n;             // forward (Y, P) per mode: [2][n]
  T* exb = exf + 2 * (size_t)n;              // backward (X, Q) per mode: [2][n]
  size_t off = (size_t)(R + 4) * n * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  DstSmem<T> sm = dst_smem_carve<T>(smem_raw + off, pl, Q);
  dst_load_tables<T>(pl, sm);

  // 1. forward DST of the local lines
  const double* src = in + (long long)(b / ib.nper) * ib.rhs_stride + ib.off[b % ib.nper];
  for (int l0 = 0; l0 < nloc; l0 += lpb) {
    const int nl = min(lpb, nloc - l0);
    __syncthreads();  // tables loaded; the previous batch's outputs have been copied out
    const int total = lpb * n;
    if (L.st == 1) {
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = idx / n, t = idx - l * n;
        sm.xin[idx] = l < nl ? dl::convert<T>(src[t + (long long)(s0 + l0 + l) * L.ss]) : T(0);
      }
    } else {
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int t = idx / lpb, l = idx - t * lpb;
        sm.xin[l * n + t] = l < nl ? dl::convert<T>(src[(long long)t * L.st + (long long)(s0 + l0 + l) * L.ss]) : T(0);
      }
    }
    __syncthreads();
    const T* y = dst_lines<T, MAXR>(pl, sm, Q);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) coef[(size_t)l0 * n + idx] = y[idx];
  }
  __syncthreads();

  // 2a. forward recurrence on the local lines, zero carry; publish (Y, P)
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    T acc = T(0), pr = T(1);
    for (int s = s0; s < s1; ++s) {
      const long long g = (long long)k * ns + s;  // tables [k][s]
      const T m = mneg[g];
      T& c = coef[(size_t)(s - s0) * n + k];
      acc = fma(m, acc, rpiv[g] * c);
      pr *= m;
      c = acc;
    }
    exf[k] = acc;
    exf[n + k] = pr;
  }
  cl.sync();
  // 2b. carry from the strips above (lower s), fix-up; backward recurrence, publish (X, Q)
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    T cin = T(0);
    for (int q = 0; q < rank; ++q) {
      const T* e = cl.map_shared_rank(exf, (unsigned)q);
      cin = fma(e[n + k], cin, e[k]);
    }
    if (cin != T(0)) {
      T qq = T(1);
      for (int s = s0; s < s1; ++s) {
        qq *= mneg[(long long)k * ns + s];
        T& c = coef[(size_t)(s - s0) * n + k];
        c = fma(qq, cin, c);
      }
    }
    T acc = T(0), pr = T(1);
    for (int s = s1 - 1; s >= s0; --s) {
      const T m = mneg[(long long)k * ns + s];
      T& c = coef[(size_t)(s - s0) * n + k];
      acc = fma(m, acc, c);
      pr *= m;
      c = acc;
    }
    exb[k] = acc;
    exb[n + k] = pr;
  }
  cl.sync();
  // 2c. carry from the strips below (higher s), fix-up
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    T cdn = T(0);
    for (int q = csz - 1; q > rank; --q) {
      const T* e = cl.map_shared_rank(exb, (unsigned)q);
      cdn = fma(e[n + k], cdn, e[k]);
    }
    if (cdn != T(0)) {
      T qq = T(1);
      for (int s = s1 - 1; s >= s0; --s) {
        qq *= mneg[(long long)k * ns + s];
        T& c = coef[(size_t)(s - s0) * n + k];
        c = fma(qq, cdn, c);
      }
    }
  }

  // 3. inverse DST of the local lines, scale, store
  To* dst = out + (long long)(b / ob.nper) * ob.rhs_stride + ob.off[b % ob.nper];
  const T scale = T(2) / T(n + 1);
  for (int l0 = 0; l0 < nloc; l0 += lpb) {
    const int nl = min(lpb, nloc - l0);
    __syncthreads();  // coef complete (first batch) / previous stores done
    for (int idx = threadIdx.x; idx < lpb * n; idx += blockDim.x)
      sm.xin[idx] = idx < nl * n ? coef[(size_t)l0 * n + idx] : T(0);
    __syncthreads();
    const T* y = dst_lines<T, MAXR>(pl, sm, Q);
    if (L.st == 1) {
      for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int l = idx / n, k = idx - l * n;
        dst[k + (long long)(s0 + l0 + l) * L.ss] = dl::convert<To>(y[idx] * scale);
      }
    } else {
      for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int k = idx / nl, l = idx - k * nl;
        dst[(long long)k * L.st + (long long)(s0 + l0 + l) * L.ss] = dl::convert<To>(y[l * n + k] * scale);
      }
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename T>
size_t fused_smem(const DstPlan& pl, int R, int Q) {
  size_t off = (size_t)(R + 4) * pl.n * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  return off + dst_smem_bytes<T>(pl.p, pl.N, Q, pl.mode);
}

// Cluster size, strip length and line batch for this block shape; false when
// the block does not fit one cluster's shared memory.
// The smallest cluster whose strips fit is widened (up to 16 CTAs, strips of at
// least 8 lines) while the grid has fewer than two CTAs per SM.
template <typename T>
bool fused_shape(const DstPlan& pl, int ns, int nblk, int* csz, int* R, int* Q) {
  const size_t budget = 200 * 1024;
  auto fit = [&](int c, int* r_out, int* q_out) {
    const int r = (ns + c - 1) / c;
    if ((size_t)r * pl.n * sizeof(T) > 112 * 1024) return false;  // coefficients of the strip
    for (int q = 4; q >= 1; --q) {
      if (2 * q > r && q > 1) continue;
      if (fused_smem<T>(pl, r, q) <= budget) {
        *r_out = r;
        *q_out = q;
        return true;
      }
    }
    return false;
  };
  int c = 1, r = 0, q = 0;
  while (c <= 16 && !fit(c, &r, &q)) c *= 2;
  if (c > 16) return false;
  while (c < 16 && (long long)nblk * c < 2 * 152 && (ns + 2 * c - 1) / (2 * c) >= 8) {
    int r2, q2;
    if (!fit(2 * c, &r2, &q2)) break;
    c *= 2;
    r = r2;
    q = q2;
  }
  *csz = c;
  *R = r;
  *Q = q;
  return true;
}

template <typename T, typename To, int MAXR>
cudaError_t launch_fused_impl(int csz, int R, int Q, const FastSolveTables& tb, LineLayout L, const double* in,
                              BatchDesc ib, To* out, BatchDesc ob, int nblk, const int* active, int nper_active,
                              cudaStream_t st) {
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_fast_solve_fused<T, To, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_fast_solve_fused<T, To, MAXR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csz, nblk, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = fused_smem<T>(tb.plan, R, Q);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fast_solve_fused<T, To, MAXR>, in, ib, out, ob, L, tb.plan, (const T*)tb.rpiv,
                            (const T*)tb.mneg, R, Q, active, nper_active);
}

}  // namespace
}  // namespace fpg
