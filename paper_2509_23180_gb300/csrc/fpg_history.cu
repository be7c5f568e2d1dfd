// Residual history of the Schur iteration (Sec. 3.2, the residual curves of the
// GMRES study): after every Arnoldi step, the GMRES residual estimate
// |g_{j+1}| of each right-hand side is copied to hist[r][iters_r - 1], where
// iters_r counts that right-hand side's steps.  A right-hand side that stopped
// iterating keeps its count and value, so the copy repeats the same entry: the
// kernel needs no knowledge of which right-hand sides were active.
#include <cuda_runtime.h>

#include "fpg_internal.cuh"

namespace fpg {
namespace {

__global__ void k_record_history(const double* __restrict__ res, const int* __restrict__ iters,
                                 double* __restrict__ hist, int len, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int i = iters[r] - 1;
  if (i >= 0 && i < len) hist[(long long)r * len + i] = res[r];
}

}  // namespace

cudaError_t launch_record_history(const double* res, const int* iters, double* hist, int len, int nrhs,
                                  cudaStream_t st) {
  k_record_history<<<(nrhs + 127) / 128, 128, 0, st>>>(res, iters, hist, len, nrhs);
  return cudaGetLastError();
}

}  // namespace fpg
