// Host side of the fused one-pass fast solve (kernel: fpg_fused_kernel.cuh,
// instantiated per radix family in fpg_fused_r*.cu).
#include <cuda_runtime.h>

#include "fpg_fused_kernel.cuh"

namespace fpg {

#define FPG_FUSED_FAMILY_DECL(R)                                                                                 \
  cudaError_t fused_family_##R(int combo, int csz, int Rl, int Q, const FastSolveTables& tb, LineLayout L,       \
                               const double* in, BatchDesc ib, void* out, BatchDesc ob, int nblk,                \
                               const int* active, int nper_active, cudaStream_t st);
FPG_FUSED_FAMILY_DECL(5)
FPG_FUSED_FAMILY_DECL(13)
FPG_FUSED_FAMILY_DECL(19)
#undef FPG_FUSED_FAMILY_DECL

namespace {

template <typename T, typename To>
cudaError_t launch_fused_typed(const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib, To* out,
                               BatchDesc ob, int nblk, const int* active, int nper_active, cudaStream_t st) {
  const DstPlan& pl = tb.plan;
  if (pl.mode == DST_DENSE) return cudaErrorNotSupported;
  int csz = 0, R = 0, Q = 0;
  if (!fused_shape<T>(pl, L.ns, nblk, &csz, &R, &Q)) return cudaErrorNotSupported;
  const int combo = sizeof(T) == 8 ? 0 : (sizeof(To) == 8 ? 1 : 2);
  switch (plan_maxr(pl)) {
    case 5: return fused_family_5(combo, csz, R, Q, tb, L, in, ib, out, ob, nblk, active, nper_active, st);
    case 13: return fused_family_13(combo, csz, R, Q, tb, L, in, ib, out, ob, nblk, active, nper_active, st);
    case 19: return fused_family_19(combo, csz, R, Q, tb, L, in, ib, out, ob, nblk, active, nper_active, st);
    default: return cudaErrorNotSupported;  // radices above 19: the three-kernel path
  }
}

}  // namespace

// Whether the fused form handles this block shape (host-side check, no launch).
bool fast_solve_fused_fits(int prec, const FastSolveTables& tb, LineLayout L) {
  int csz, R, Q;
  if (tb.plan.mode == DST_DENSE || plan_maxr(tb.plan) > 19) return false;
  return prec == 64 ? fused_shape<double>(tb.plan, L.ns, 1, &csz, &R, &Q)
                    : fused_shape<float>(tb.plan, L.ns, 1, &csz, &R, &Q);
}

cudaError_t launch_fast_solve_fused(int prec, int out_prec, const FastSolveTables& tb, LineLayout L,
                                    const double* in, BatchDesc ib, void* out, BatchDesc ob, int nblk,
                                    const int* active, int nper_active, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  if (prec == 64)
    return launch_fused_typed<double, double>(tb, L, in, ib, (double*)out, ob, nblk, active, nper_active, st);
  if (out_prec == 64)
    return launch_fused_typed<float, double>(tb, L, in, ib, (double*)out, ob, nblk, active, nper_active, st);
  return launch_fused_typed<float, float>(tb, L, in, ib, (float*)out, ob, nblk, active, nper_active, st);
}

}  // namespace fpg
