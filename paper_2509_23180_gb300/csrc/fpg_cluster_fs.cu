// One-pass FP32 fast solve z = A^{-1} v of the centre block (Sec. 2.1: DST-I
// along x, one tridiagonal solve per mode along y, inverse DST-I), for the
// block lengths whose line DST is compiled (p = n + 1 = 65 and 513): each block
// is read once from HBM (FP64) and written once (FP32 or FP64), with nothing in
// between in global memory.
//
// One thread-block cluster per block.  CTA r of the C = n / R CTAs owns the R
// consecutive lines (rows) s0 = r R .. s0 + R - 1 and keeps their spectral
// coefficients in its shared memory as a strip [R][n+1] for the whole solve:
//   1. load the strip (FP64 -> FP32 on the integer pipe) and apply the line DST
//      in place, 2Q lines at a time, with the size-specialised engine
//      (fpg_dstline_impl.cuh: pack, two-pass DFT of length p, unpack);
//   2. the tridiagonal solve of every mode k across the cluster.  The pivots
//      are generated in the strip, not read from a table: with sigma_k =
//      4 sin^2(k pi / 2p) - kappa / delta and the scaled pivot
//      w_s = -(u_s / delta) - 1 of tridiag(delta, d_k, delta), the LU recurrence
//      u_s = d_k - delta^2 / u_{s-1} becomes
//          w_0 = 1 + sigma_k,   w_s = sigma_k + w_{s-1} / (1 + w_{s-1}),
//      a sum of positive terms (no cancellation, so FP32 keeps full relative
//      precision even in the lowest modes, where u_s is -2 delta plus a small
//      part), and the multiplier m_s = -delta / u_s = 1 / (1 + w_s).  The
//      forward sweep on f' = f is y_s = m_s (y_{s-1} + f_s) (the exact sweep
//      on -f/delta, scaled by -delta; the -1/delta is folded into the output
//      scale) and the back substitution x_s = y_s + m_s x_{s+1}.  Each CTA runs
//      both recurrences on its rows with a zero carry; the carries are linear,
//      so the true values follow from the products of m over the strips: the
//      CTAs publish (end value, product) per mode in shared memory, and after a
//      cluster barrier every CTA folds those of the CTAs before it (forward) or
//      after it (backward) through distributed shared memory and fixes up its
//      rows.  w at each strip start comes from a small host table (FP64
//      recurrence, rounded once).
//   3. the inverse DST of the strip in place, scaled by 2/p (with the two
//      unpacking factors 1/2 and the -1/delta), stored.
// Work per point as the three-kernel path; HBM traffic 8 B in + 4 B (FP32) or
// 8 B (FP64) out per point, the algorithmic minimum.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fpg_dstline_impl.cuh"
#include "fpg_host_tables.h"
#include "fpg_internal.cuh"

namespace fpg {
namespace {

template <int P>
struct ClusterShape {
  using S = dl::LineShape<float, P>;
  static constexpr int n = P - 1, R = kClusterRows, Q = S::Q, NT = S::NT, LP = S::LP;
  static constexpr int C = n / R;          // CTAs per cluster (one block)
  static constexpr int CH = R / (2 * Q);   // DST batches of 2Q lines per strip
  static_assert(!S::rader, "the in-place strip needs the spectra to overlay their lines (non-Rader plans)");
  static_assert(n % R == 0 && R % (2 * Q) == 0 && C >= 1 && C <= 16, "strip shape");
  static constexpr size_t o_strip = S::o_lines;  // after the DST tables (sin, twiddles, dc)
  static constexpr size_t o_y = dl::align16(o_strip + sizeof(float) * R * LP);
  static constexpr size_t o_ex = dl::align16(o_y + sizeof(C2<float>) * Q * S::A * S::YB);
  static constexpr size_t bytes = dl::align16(o_ex + sizeof(float) * 3 * n);
};

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  cluster_arrive_release();
  cluster_wait_acquire();
}

// Multipliers m_s of mode k on the strip's rows, from the scaled pivot w at the
// strip start: m_i = 1 / (1 + w_i), w_{i+1} = sigma + w_i m_i.
template <int R>
__device__ __forceinline__ void strip_multipliers(float w, float sig, float (&m)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    m[i] = __frcp_rn(1.0f + w);
    w = fmaf(w, m[i], sig);
  }
}

// blocks: n x n, rows contiguous (x fastest), block b at in + boff(ib, b) and
// out + boff(ob, b), both 16-byte aligned; grid (C, nblk), cluster (C, 1, 1).
template <int P, typename To>
__global__ void __launch_bounds__(dl::LineShape<float, P>::NT, 2)
k_fast_solve_cluster(const double* __restrict__ in, BatchDesc ib, To* __restrict__ out, BatchDesc ob, DstPlan pl,
                     const float* __restrict__ sigma, const float* __restrict__ wseed, float scale,
                     const int* __restrict__ active, int nper_active) {
  using CS = ClusterShape<P>;
  using S = typename CS::S;
  constexpr int n = CS::n, R = CS::R, Q = CS::Q, NT = CS::NT, LP = CS::LP, C = CS::C;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;  // the same b for the whole cluster
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dl::LineSmem<float, P> s(smem_raw);
  float* strip = reinterpret_cast<float*>(smem_raw + CS::o_strip);  // [R][LP]
  s.y = reinterpret_cast<C2<float>*>(smem_raw + CS::o_y);
  float* ex = reinterpret_cast<float*>(smem_raw + CS::o_ex);  // [3][n]: forward end, product, backward start
  dl::load_tables<float, P>(pl, s);

  // 1. load the strip: R contiguous rows of FP64, 8 two-element loads in flight per thread
  {
    const double2* src = reinterpret_cast<const double2*>(in + dl::boff(ib, b) + (long long)rank * R * n);
    constexpr int TOT = R * n / 2, U = 8;
    for (int base = 0; base < TOT; base += NT * U) {
      double2 v[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = base + j * NT + (int)threadIdx.x;
        v[j] = i < TOT ? src[i] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = base + j * NT + (int)threadIdx.x;
        if (i < TOT) {
          const int l = i / (n / 2), t2 = i - l * (n / 2);
          strip[l * LP + 2 * t2] = dl::convert<float>(v[j].x);
          strip[l * LP + 2 * t2 + 1] = dl::convert<float>(v[j].y);
        }
      }
    }
  }
  __syncthreads();
  // forward DST of the strip in place (spectra overlay their own pair of lines)
#pragma unroll 1
  for (int c = 0; c < CS::CH; ++c) {
    s.lines = strip + c * 2 * Q * LP;
    s.x = reinterpret_cast<C2<float>*>(s.lines);
    dl::unpack<float, P>(s, dl::dft_p<float, P>(s));
    __syncthreads();
  }

  // 2. tridiagonal solve of every mode across the cluster
  for (int k = threadIdx.x; k < n; k += NT) {
    float m[R];
    strip_multipliers<R>(wseed[rank * n + k], sigma[k], m);
    float acc = 0.0f, pr = 1.0f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      float* c = strip + i * LP + k;
      acc = m[i] * (acc + *c);
      pr *= m[i];
      *c = acc;
    }
    ex[k] = acc;      // forward value at the strip's last row (zero carry in)
    ex[n + k] = pr;   // product of the strip's multipliers
  }
  cluster_sync_all();
  for (int k = threadIdx.x; k < n; k += NT) {
    float cin = 0.0f;  // y at the row before the strip: fold of the strips before it
#pragma unroll
    for (int q = 0; q < C; ++q) {
      if (q < (int)rank) {
        const float* e = cl.map_shared_rank(ex, (unsigned)q);
        cin = fmaf(e[n + k], cin, e[k]);
      }
    }
    float m[R];
    strip_multipliers<R>(wseed[rank * n + k], sigma[k], m);
    if (cin != 0.0f) {
      float pp = 1.0f;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        pp *= m[i];
        float* c = strip + i * LP + k;
        *c = fmaf(pp, cin, *c);
      }
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
      float* c = strip + i * LP + k;
      acc = fmaf(m[i], acc, *c);
      *c = acc;
    }
    ex[2 * n + k] = acc;  // back substitution at the strip's first row (zero carry from above)
  }
  cluster_sync_all();
  for (int k = threadIdx.x; k < n; k += NT) {
    float xt = 0.0f;  // x at the row after the strip: fold of the strips after it
#pragma unroll
    for (int q = C - 1; q >= 0; --q) {
      if (q > (int)rank) {
        const float* e = cl.map_shared_rank(ex, (unsigned)q);
        xt = fmaf(e[n + k], xt, e[2 * n + k]);
      }
    }
    if (xt != 0.0f) {
      float m[R];
      strip_multipliers<R>(wseed[rank * n + k], sigma[k], m);
      float qq = 1.0f;
#pragma unroll
      for (int i = R - 1; i >= 0; --i) {
        qq *= m[i];
        float* c = strip + i * LP + k;
        *c = fmaf(qq, xt, *c);
      }
    }
  }
  // the other CTAs may still read this CTA's ex: arrive now, wait before leaving
  cluster_arrive_release();
  __syncthreads();

  // 3. inverse DST in place, scale, store
  To* dst = out + dl::boff(ob, b) + (long long)rank * R * n;
#pragma unroll 1
  for (int c = 0; c < CS::CH; ++c) {
    s.lines = strip + c * 2 * Q * LP;
    s.x = reinterpret_cast<C2<float>*>(s.lines);
    dl::unpack<float, P>(s, dl::dft_p<float, P>(s));
    __syncthreads();
    To* d = dst + (long long)c * 2 * Q * n;
    for (int i = threadIdx.x; i < 2 * Q * (n / 2); i += NT) {
      const int l = i / (n / 2), t2 = i - l * (n / 2);
      const float a0 = s.lines[l * LP + 2 * t2] * scale, a1 = s.lines[l * LP + 2 * t2 + 1] * scale;
      if constexpr (sizeof(To) == 8) {
        reinterpret_cast<double2*>(d)[i] = make_double2(dl::convert<double>(a0), dl::convert<double>(a1));
      } else {
        reinterpret_cast<float2*>(d)[i] = make_float2(a0, a1);
      }
    }
  }
  cluster_wait_acquire();
}

template <int P, typename To>
cudaError_t launch_cluster_p(const FastSolveTables& tb, const double* in, BatchDesc ib, To* out, BatchDesc ob,
                             int nblk, const int* active, int nper_active, cudaStream_t st) {
  using CS = ClusterShape<P>;
  auto kern = k_fast_solve_cluster<P, To>;
  static PerDeviceOnce attr;
  static int fits[64] = {};  // per device: 1 a cluster of this shape can be resident, -1 it cannot
  int dev = 0;
  cudaGetDevice(&dev);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS::C, (unsigned)nblk, 1);
  cfg.blockDim = dim3(CS::NT, 1, 1);
  cfg.dynamicSmemBytes = CS::bytes;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CS::bytes);
    if (CS::C > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int clusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (dev >= 0 && dev < 64) fits[dev] = (e == cudaSuccess && clusters > 0) ? 1 : -1;
    cudaGetLastError();
  }
  if (dev >= 0 && dev < 64 && fits[dev] < 0) return cudaErrorNotSupported;
  // scale: 2/p for the transform pair, 1/4 for the two unpacking factors, -1/delta for the sweep's scaling
  const double delta = tb.delta;
  const float scale = (float)((2.0 / P) * 0.25 * (-1.0 / delta));
  return cudaLaunchKernelEx(&cfg, kern, in, ib, out, ob, tb.plan, (const float*)tb.cl_sigma,
                            (const float*)tb.cl_wseed, scale, active, nper_active);
}

bool aligned16(const void* p, const BatchDesc& d, size_t esize) {
  if (reinterpret_cast<uintptr_t>(p) % 16) return false;
  if ((d.rhs_stride * (long long)esize) % 16) return false;
  for (int i = 0; i < d.nper; ++i)
    if ((d.off[i] * (long long)esize) % 16) return false;
  return true;
}

}  // namespace

// Can the one-pass cluster kernel take this FP32 fast solve?  The centre block's
// layout (n x n, rows contiguous), a compiled length (p = 65 or 513), the
// tables present, and 16-byte aligned blocks.
bool fast_solve_cluster_fits(const FastSolveTables& tb, LineLayout L) {
  const int p = tb.plan.p;
  if (p != 65 && p != 513) return false;
  if (tb.kind != 0 || tb.cl_sigma == nullptr || tb.cl_wseed == nullptr) return false;
  return L.st == 1 && L.ss == L.nt && L.nt == tb.n && L.ns == tb.n;
}

cudaError_t launch_fast_solve_cluster(int out_prec, const FastSolveTables& tb, LineLayout L, const double* in,
                                      BatchDesc ib, void* out, BatchDesc ob, int nblk, const int* active,
                                      int nper_active, cudaStream_t st) {
  if (!fast_solve_cluster_fits(tb, L)) return cudaErrorNotSupported;
  if (!aligned16(in, ib, 8) || !aligned16(out, ob, out_prec == 64 ? 8 : 4)) return cudaErrorNotSupported;
  const int p = tb.plan.p;
  if (out_prec == 64) {
    return p == 65 ? launch_cluster_p<65, double>(tb, in, ib, (double*)out, ob, nblk, active, nper_active, st)
                   : launch_cluster_p<513, double>(tb, in, ib, (double*)out, ob, nblk, active, nper_active, st);
  }
  return p == 65 ? launch_cluster_p<65, float>(tb, in, ib, (float*)out, ob, nblk, active, nper_active, st)
                 : launch_cluster_p<513, float>(tb, in, ib, (float*)out, ob, nblk, active, nper_active, st);
}


}  // namespace fpg
