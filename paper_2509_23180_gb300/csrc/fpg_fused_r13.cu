// One radix family (MAXR = 13) of the fused one-pass fast-solve kernel; the
// families compile as separate translation units so that the build runs them
// in parallel.
#include "fpg_fused_kernel.cuh"

namespace fpg {

cudaError_t fused_family_13(int combo, int csz, int R, int Q, const FastSolveTables& tb, LineLayout L,
                            const double* in, BatchDesc ib, void* out, BatchDesc ob, int nblk, const int* active,
                            int nper_active, cudaStream_t st) {
  switch (combo) {
    case 0:
      return launch_fused_impl<double, double, 13>(csz, R, Q, tb, L, in, ib, (double*)out, ob, nblk, active,
                                                   nper_active, st);
    case 1:
      return launch_fused_impl<float, double, 13>(csz, R, Q, tb, L, in, ib, (double*)out, ob, nblk, active,
                                                  nper_active, st);
    default:
      return launch_fused_impl<float, float, 13>(csz, R, Q, tb, L, in, ib, (float*)out, ob, nblk, active,
                                                 nper_active, st);
  }
}

}  // namespace fpg
