// Radix family MAXR = 43 of the generic-engine DST kernels, FP64 part (the FP32
// part is in fpg_fft_r43f.cu: this family is the slowest to compile).
#include "fpg_fft_kernels.cuh"

namespace fpg {

cudaError_t fft_family_fwd_43f(dim3 grid, size_t smem, cudaStream_t st, const double* in, BatchDesc ib, LineLayout L,
                               const DstPlan& pl, void* scratch, int Q, const int* active, int nper_active);
cudaError_t fft_family_inv_43f(int out_prec, dim3 grid, size_t smem, cudaStream_t st, const void* scratch, void* out,
                               BatchDesc ob, LineLayout L, const DstPlan& pl, int Q, const int* active,
                               int nper_active);

cudaError_t fft_family_fwd_43(int prec, dim3 grid, size_t smem, cudaStream_t st, const double* in, BatchDesc ib,
                              LineLayout L, const DstPlan& pl, void* scratch, int Q, const int* active,
                              int nper_active) {
  if (prec == 64)
    return fft_fwd_launch<double, 43>(grid, smem, st, in, ib, L, pl, (double*)scratch, Q, active, nper_active);
  return fft_family_fwd_43f(grid, smem, st, in, ib, L, pl, scratch, Q, active, nper_active);
}

cudaError_t fft_family_inv_43(int prec, int out_prec, dim3 grid, size_t smem, cudaStream_t st, const void* scratch,
                              void* out, BatchDesc ob, LineLayout L, const DstPlan& pl, int Q, const int* active,
                              int nper_active) {
  if (prec == 64)
    return fft_inv_launch<double, double, 43>(grid, smem, st, (const double*)scratch, (double*)out, ob, L, pl, Q,
                                              active, nper_active);
  return fft_family_inv_43f(out_prec, grid, smem, st, scratch, out, ob, L, pl, Q, active, nper_active);
}

}  // namespace fpg
