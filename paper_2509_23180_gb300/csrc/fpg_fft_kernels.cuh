// Generic-engine DST kernels of the fast solve (any n with an FFT plan), one
// template per radix family; instantiated in fpg_fft_r*.cu so that the
// families compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"

namespace fpg {
namespace {

constexpr int kFftThreads = 256;

__device__ __forceinline__ const double* fft_batch_ptr(const double* base, const BatchDesc& d, int b) {
  return base + (long long)(b / d.nper) * d.rhs_stride + d.off[b % d.nper];
}
template <typename To>
__device__ __forceinline__ To* fft_batch_ptr_out(To* base, const BatchDesc& d, int b) {
  return base + (long long)(b / d.nper) * d.rhs_stride + d.off[b % d.nper];
}

// FFT engine versions: 2Q lines per CTA.
template <typename T, int MAXR>
__global__ void __launch_bounds__(kFftThreads)
k_fft_forward(const double* __restrict__ in, BatchDesc ib, LineLayout L, DstPlan pl, T* __restrict__ scratch,
              int Q, const int* __restrict__ active, int nper_active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  const int n = pl.n;
  const int lpb = 2 * Q;
  const int s0 = blockIdx.x * lpb;
  const int nl = min(lpb, L.ns - s0);
  DstSmem<T> sm = dst_smem_carve<T>(smem_raw, pl, Q);
  dst_load_tables<T>(pl, sm);
  const double* src = fft_batch_ptr(in, ib, b);
  const int total = lpb * n;
  if (L.st == 1) {
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int l = idx / n, t = idx - l * n;
      sm.xin[idx] = l < nl ? dl::convert<T>(src[t + (long long)(s0 + l) * L.ss]) : T(0);
    }
  } else {
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int t = idx / lpb, l = idx - t * lpb;
      sm.xin[l * n + t] = l < nl ? dl::convert<T>(src[(long long)t * L.st + (long long)(s0 + l) * L.ss]) : T(0);
    }
  }
  __syncthreads();
  const T* y = dst_lines<T, MAXR>(pl, sm, Q);
  // scratch[b][k][s]: l fastest, so a warp writes runs of nl consecutive rows
  T* dst = scratch + (long long)b * n * L.ns + s0;
  for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
    const int k = idx / nl, l = idx - k * nl;
    dst[(long long)k * L.ns + l] = y[l * n + k];
  }
}

template <typename T, typename To, int MAXR>
__global__ void __launch_bounds__(kFftThreads)
k_fft_inverse(const T* __restrict__ scratch, To* __restrict__ out, BatchDesc ob, LineLayout L, DstPlan pl, int Q,
              const int* __restrict__ active, int nper_active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  const int n = pl.n;
  const int lpb = 2 * Q;
  const int s0 = blockIdx.x * lpb;
  const int nl = min(lpb, L.ns - s0);
  DstSmem<T> sm = dst_smem_carve<T>(smem_raw, pl, Q);
  dst_load_tables<T>(pl, sm);
  const T* src = scratch + (long long)b * n * L.ns + s0;  // [b][k][s]
  for (int idx = threadIdx.x; idx < lpb * n; idx += blockDim.x) {
    const int k = idx / lpb, l = idx - k * lpb;
    sm.xin[l * n + k] = l < nl ? src[(long long)k * L.ns + l] : T(0);
  }
  __syncthreads();
  const T* y = dst_lines<T, MAXR>(pl, sm, Q);
  To* dst = fft_batch_ptr_out(out, ob, b);
  const T scale = T(2) / T(n + 1);
  if (L.st == 1) {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int l = idx / n, k = idx - l * n;
      dst[k + (long long)(s0 + l) * L.ss] = dl::convert<To>(y[idx] * scale);
    }
  } else {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int k = idx / nl, l = idx - k * nl;
      dst[(long long)k * L.st + (long long)(s0 + l) * L.ss] = dl::convert<To>(y[l * n + k] * scale);
    }
  }
}


template <typename T, int MAXR>
cudaError_t fft_fwd_launch(dim3 grid, size_t smem, cudaStream_t st, const double* in, BatchDesc ib, LineLayout L,
                           const DstPlan& pl, T* scratch, int Q, const int* active, int nper_active) {
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_fft_forward<T, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  k_fft_forward<T, MAXR><<<grid, kFftThreads, smem, st>>>(in, ib, L, pl, scratch, Q, active, nper_active);
  return cudaGetLastError();
}

template <typename T, typename To, int MAXR>
cudaError_t fft_inv_launch(dim3 grid, size_t smem, cudaStream_t st, const T* scratch, To* out, BatchDesc ob,
                           LineLayout L, const DstPlan& pl, int Q, const int* active, int nper_active) {
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_fft_inverse<T, To, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  k_fft_inverse<T, To, MAXR><<<grid, kFftThreads, smem, st>>>(scratch, out, ob, L, pl, Q, active, nper_active);
  return cudaGetLastError();
}

}  // namespace
}  // namespace fpg
