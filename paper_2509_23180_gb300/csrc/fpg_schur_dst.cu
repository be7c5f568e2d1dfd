// a2, reduced interface correction by transforms: for C's line next to arm a,
//   corr_a = delta^2 Q diag(g_k) Q line_a,  Q = sqrt(2/(n+1)) DST-I,
// with g_k = [T_k^{-1}]_{N,N} the last reciprocal Thomas pivot of the arm's
// mode-k system (N = n + 1, Eq. "trans_subeq" on the arm).  This is the same
// operator as the Toeplitz-minus-Hankel sum of k_schur_lines, applied with two
// DST-I of length n per line (O(n log n) instead of O(n^2)) through the
// size-specialised line DST engine.  The engine's transform is 2 * DST-I, so
// the scale between the two transforms is g_k delta^2 / (2 (n+1)).
#include <cuda_runtime.h>

#include "fpg_dstline_impl.cuh"

namespace fpg {
namespace {

template <typename Tz>
__device__ __forceinline__ double facing_line(const Tz* z, int n, int a, int q) {
  long long i;
  switch (a) {
    case 0: i = (long long)q * n; break;                // x = h column (W)
    case 1: i = (long long)q * n + n - 1; break;        // x = 1 - h column (E)
    case 2: i = q; break;                               // y = h row (S)
    default: i = (long long)(n - 1) * n + q; break;     // y = 1 - h row (N)
  }
  return dl::convert<double>(z[i]);
}

template <int P, typename Tz>
__global__ void __launch_bounds__(dl::LineShape<double, P>::NT)
k_schur_lines_dst(const Tz* __restrict__ z, long long zstride, DstPlan pl, const double* __restrict__ gsc,
                  const int* __restrict__ arms, int narms, double* __restrict__ corr, const int* __restrict__ active,
                  int nlines) {
  using S = dl::LineShape<double, P>;
  constexpr int n = S::n, Q = S::Q, NT = S::NT, LP = S::LP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dl::LineSmem<double, P> s(smem_raw);
  dl::load_tables<double, P>(pl, s);
  const int l0 = blockIdx.x * 2 * Q;
  for (int i = threadIdx.x; i < 2 * Q * n; i += NT) {
    const int l = i / n, t = i - l * n;
    const int g = l0 + l;
    double v = 0.0;
    if (g < nlines) {
      const int r = g / narms, a = arms[g - r * narms];
      if (active == nullptr || active[r]) v = facing_line(z + (long long)r * zstride, n, a, t);
    }
    s.lines[l * LP + t] = v;
  }
  __syncthreads();
  dl::unpack<double, P>(s, dl::dft_p<double, P>(s));
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * Q * n; i += NT) {
    const int l = i / n, k = i - l * n;
    s.lines[l * LP + k] *= gsc[k];
  }
  __syncthreads();
  dl::unpack<double, P>(s, dl::dft_p<double, P>(s));
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * Q * n; i += NT) {
    const int l = i / n, k = i - l * n;
    const int g = l0 + l;
    if (g >= nlines) continue;
    const int r = g / narms, a = arms[g - r * narms];
    if (active != nullptr && !active[r]) continue;
    corr[((long long)r * 4 + a) * n + k] = s.lines[l * LP + k];
  }
}

template <int P>
cudaError_t schur_dst_one(const void* z, int zprec, long long zstride, const DstPlan& pl, const double* gsc,
                          const int* arms, int narms, double* corr, const int* active, int nrhs, cudaStream_t st) {
  using S = dl::LineShape<double, P>;
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_schur_lines_dst<P, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    cudaFuncSetAttribute(k_schur_lines_dst<P, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
  }
  const int nlines = nrhs * narms;
  const dim3 grid((nlines + 2 * S::Q - 1) / (2 * S::Q));
  if (zprec == 64)
    k_schur_lines_dst<P, double><<<grid, S::NT, S::bytes, st>>>((const double*)z, zstride, pl, gsc, arms, narms, corr,
                                                               active, nlines);
  else
    k_schur_lines_dst<P, float><<<grid, S::NT, S::bytes, st>>>((const float*)z, zstride, pl, gsc, arms, narms, corr,
                                                              active, nlines);
  return cudaGetLastError();
}

}  // namespace

bool schur_dst_supported(int n) { return n == 64 || n == 256 || n == 512; }

// FP64 plan of length n (the centre block's); gsc[k] = g_k delta^2 / (2 (n+1)).
cudaError_t launch_schur_dst(const void* z, int zprec, long long zstride, int n, const DstPlan& pl, const double* gsc,
                             const int* arms, int narms, double* corr, const int* active, int nrhs, cudaStream_t st) {
  switch (n) {
    case 64: return schur_dst_one<65>(z, zprec, zstride, pl, gsc, arms, narms, corr, active, nrhs, st);
    case 256: return schur_dst_one<257>(z, zprec, zstride, pl, gsc, arms, narms, corr, active, nrhs, st);
    case 512: return schur_dst_one<513>(z, zprec, zstride, pl, gsc, arms, narms, corr, active, nrhs, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace fpg
