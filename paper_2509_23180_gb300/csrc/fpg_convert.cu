// fpg_convert: element-wise binary64 <-> binary32 conversion with the
// integer-pipe routines of the mixed-precision path (the FP32 preconditioner
// reads FP64 basis vectors and the FP64 Schur matvec reads FP32 z).
#include <cuda_runtime.h>

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"

namespace fpg {

void record_message(const char* msg);

namespace {

__global__ void k_convert_d2f(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = dl::f64_to_f32(in[i]);
}

__global__ void k_convert_f2d(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = dl::f32_to_f64(in[i]);
}

}  // namespace
}  // namespace fpg

extern "C" fpg_status fpg_convert(const void* in, int32_t in_prec, void* out, int32_t out_prec, int64_t count,
                                  void* stream) {
  using namespace fpg;
  if (!in || !out || count < 0 || (in_prec != 32 && in_prec != 64) || (out_prec != 32 && out_prec != 64) ||
      in_prec == out_prec) {
    record_message("fpg_convert: null pointer, negative count or precisions not one of (64, 32) / (32, 64)");
    return FPG_EINVAL;
  }
  if (count == 0) return FPG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256;
  const long long want = (count + threads - 1) / threads;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  if (in_prec == 64)
    k_convert_d2f<<<blocks, threads, 0, st>>>((const double*)in, (float*)out, count);
  else
    k_convert_f2d<<<blocks, threads, 0, st>>>((const float*)in, (double*)out, count);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    record_cuda_error(e, "fpg_convert");
    return FPG_ECUDA;
  }
  return FPG_OK;
}
