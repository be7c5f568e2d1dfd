// Radix family MAXR = 13 of the generic-engine DST kernels.
#include "fpg_fft_kernels.cuh"

namespace fpg {

cudaError_t fft_family_fwd_13(int prec, dim3 grid, size_t smem, cudaStream_t st, const double* in, BatchDesc ib,
                              LineLayout L, const DstPlan& pl, void* scratch, int Q, const int* active,
                              int nper_active) {
  if (prec == 64)
    return fft_fwd_launch<double, 13>(grid, smem, st, in, ib, L, pl, (double*)scratch, Q, active, nper_active);
  return fft_fwd_launch<float, 13>(grid, smem, st, in, ib, L, pl, (float*)scratch, Q, active, nper_active);
}

cudaError_t fft_family_inv_13(int prec, int out_prec, dim3 grid, size_t smem, cudaStream_t st, const void* scratch,
                              void* out, BatchDesc ob, LineLayout L, const DstPlan& pl, int Q, const int* active,
                              int nper_active) {
  if (prec == 64)
    return fft_inv_launch<double, double, 13>(grid, smem, st, (const double*)scratch, (double*)out, ob, L, pl, Q,
                                              active, nper_active);
  if (out_prec == 64)
    return fft_inv_launch<float, double, 13>(grid, smem, st, (const float*)scratch, (double*)out, ob, L, pl, Q,
                                             active, nper_active);
  return fft_inv_launch<float, float, 13>(grid, smem, st, (const float*)scratch, (float*)out, ob, L, pl, Q, active,
                                          nper_active);
}

}  // namespace fpg
