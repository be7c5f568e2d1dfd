// Size-specialised line DST kernels, FP64 compute.
#include "fpg_dstline_impl.cuh"

namespace fpg {

bool dst_lines_supported_f64(int p) { return p == 65 || p == 257 || p == 513; }

// The specialised kernels run one thread (p = 257 in FP64: one quad of four)
// per sub-DFT, (lines / 2) * A threads per pass.  FP64 needs enough of them to keep the FP64 pipe busy: 10
// blocks of 256^2 (20480 threads) are already faster than the generic engine
// (84 / 74 us against 91 / 88 us per forward / inverse launch); a single 64^2
// block (416 threads) stays on the generic engine.
bool dst_lines_profitable_f64(int p, int nblk, int ns) {
  int ab = 0;
  switch (p) {
    case 65: ab = dl::LineCfg<double, 65>::A; break;
    case 257: ab = dl::LineCfg<double, 257>::A * (dl::LineQuad<double, 257>::value ? 4 : 1); break;
    case 513: ab = dl::LineCfg<double, 513>::A; break;
    default: return false;
  }
  return (long long)nblk * ((ns + 1) / 2) * ab >= 10000;
}

cudaError_t dst_lines_fwd_f64(int p, const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl,
                              double* scratch, int nblk, const int* active, int nper_active, int vec,
                              cudaStream_t st) {
  switch (p) {
    case 65: return dl::fwd_one<double, 65>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    case 257: return dl::fwd_one<double, 257>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    case 513: return dl::fwd_one<double, 513>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t dst_lines_inv_f64(int p, const double* scratch, double* out, BatchDesc ob, LineLayout L,
                              const DstPlan& pl, int nblk, const int* active, int nper_active, int vec,
                              cudaStream_t st) {
  switch (p) {
    case 65: return dl::inv_one<double, double, 65>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    case 257: return dl::inv_one<double, double, 257>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    case 513: return dl::inv_one<double, double, 513>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace fpg
