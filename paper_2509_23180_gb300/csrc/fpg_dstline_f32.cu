// Size-specialised line DST kernels, FP32 compute (FP64 input, FP32 or FP64 output).
#include "fpg_dstline_impl.cuh"

namespace fpg {

bool dst_lines_supported_f32(int p) { return p == 65 || p == 257 || p == 513 || p == 1025; }

// Status word of callers that pass none: set by the persistent forward kernel
// when a bulk-copy wait runs out.  A domain passes its own word instead, and
// its solve then returns FPG_ETIMEOUT.
__device__ int g_dst_bulk_timeout_f32 = 0;

cudaError_t dst_lines_fwd_bulk_f32(int p, const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl,
                                   float* scratch, int nblk, const int* active, int nper_active, int* err,
                                   int wait_limit, cudaStream_t st) {
  if (err == nullptr) {
    cudaError_t e = cudaGetSymbolAddress((void**)&err, g_dst_bulk_timeout_f32);
    if (e != cudaSuccess) return e;
  }
  switch (p) {
    case 65: return dl::fwd_bulk_one<float, 65>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    case 257: return dl::fwd_bulk_one<float, 257>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    case 513: return dl::fwd_bulk_one<float, 513>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    case 1025:
      return dl::fwd_bulk_one<float, 1025>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    default: return cudaErrorNotSupported;
  }
}

// The streaming forward form (k_dst_lines_fwd_stream) for this p and sweep length:
// p without Rader, ns a whole number of tiles of 2Q rows, and a measured gain over
// one CTA per tile (64 x 512^2: 76.5 against 81.9 us; 16 x 1024^2: 103 against 113;
// at p = 65 it was slower, 88 against 80, so that length keeps the per-tile kernel).
bool dst_lines_stream_ok_f32(int p, int ns) {
  switch (p) {
    case 513: return dl::StreamShape<513>::eligible && ns % (2 * dl::LineShape<float, 513>::Q) == 0;
    case 1025: return dl::StreamShape<1025>::eligible && ns % (2 * dl::LineShape<float, 1025>::Q) == 0;
    default: return false;
  }
}

cudaError_t dst_lines_fwd_stream_f32(int p, const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl,
                                     float* scratch, int nblk, const int* active, int nper_active, int* err,
                                     int wait_limit, cudaStream_t st) {
  if (err == nullptr) {
    cudaError_t e = cudaGetSymbolAddress((void**)&err, g_dst_bulk_timeout_f32);
    if (e != cudaSuccess) return e;
  }
  switch (p) {
    case 65: return dl::fwd_stream_one<65>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    case 513: return dl::fwd_stream_one<513>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    case 1025: return dl::fwd_stream_one<1025>(in, ib, L, pl, scratch, nblk, active, nper_active, err, wait_limit, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t dst_lines_fwd_f32(int p, const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl, float* scratch,
                              int nblk, const int* active, int nper_active, int vec, cudaStream_t st) {
  switch (p) {
    case 65: return dl::fwd_one<float, 65>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    case 257: return dl::fwd_one<float, 257>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    case 513: return dl::fwd_one<float, 513>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    case 1025: return dl::fwd_one<float, 1025>(in, ib, L, pl, scratch, nblk, active, nper_active, vec, st);
    default: return cudaErrorNotSupported;
  }
}

template <typename To>
static cudaError_t inv_f32(int p, const float* scratch, To* out, BatchDesc ob, LineLayout L, const DstPlan& pl,
                           int nblk, const int* active, int nper_active, int vec, cudaStream_t st) {
  switch (p) {
    case 65: return dl::inv_one<float, To, 65>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    case 257: return dl::inv_one<float, To, 257>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    case 513: return dl::inv_one<float, To, 513>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    case 1025: return dl::inv_one<float, To, 1025>(scratch, out, ob, L, pl, nblk, active, nper_active, vec, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t dst_lines_inv_f32(int p, const float* scratch, void* out, int out_prec, BatchDesc ob, LineLayout L,
                              const DstPlan& pl, int nblk, const int* active, int nper_active, int vec,
                              cudaStream_t st) {
  if (out_prec == 64)
    return inv_f32<double>(p, scratch, (double*)out, ob, L, pl, nblk, active, nper_active, vec, st);
  return inv_f32<float>(p, scratch, (float*)out, ob, L, pl, nblk, active, nper_active, vec, st);
}

}  // namespace fpg
