// fpg_fast_solve_noalloc: the fast solve z = A^{-1} v on n x n Dirichlet
// squares (the centre block's operator) for callers that cannot allocate device
// memory -- code that runs where cudaMalloc is not allowed or must not be
// called (inside another framework's memory pool, on a path whose device memory
// was fixed up front, or while the allocator is unavailable), and that cannot
// provide the workspace fpg_create_domain needs.
//
// Everything the kernels need lives in one file-scope device array of fixed
// size, g_noalloc_scratch (kNoAllocBytes, ~20 MiB): the spectral coefficients
// of the batch and the DST / Thomas tables of the last (n, kappa).  Every GPU
// that loads the library holds this array until the process exits.  Host-side
// tables are built in file-scope static arrays: no heap allocation either.
//
// The kernels are the library's fast-solve kernels (forward DST, scanned
// Thomas, inverse DST) with the scratch pointer set to this array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fpg_host_tables.h"
#include "fpg_internal.cuh"

namespace fpg {
cudaError_t launch_fast_solve(int prec, int out_prec, const FastSolveTables& tb, LineLayout L, const double* in,
                              BatchDesc ib, void* out, BatchDesc ob, int nblk, void* scratch, const int* active,
                              int nper_active, cudaStream_t st, int* launches, cudaEvent_t* ev = nullptr);
void record_message(const char* msg);
}  // namespace fpg

namespace {

using namespace fpg;

constexpr int kMaxN = FPG_NOALLOC_MAX_N;                          // largest n accepted
constexpr long long kCoeffDoubles = FPG_NOALLOC_MAX_POINTS;       // nvec * n * n limit
constexpr long long kTableDoubles = 2LL * kMaxN * kMaxN + 8LL * (kMaxN + 1) + 256;
constexpr long long kTableInts = 2LL * kMaxN + 64;
constexpr size_t kNoAllocBytes = (size_t)(kCoeffDoubles + kTableDoubles) * 8 + (size_t)kTableInts * 4 + 4096;

// The scratch array.  In host code this name is a host-side stand-in, not a
// device address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host staging for the tables (file-scope, no heap).
static double h_rpiv[kMaxN * kMaxN], h_mneg[kMaxN * kMaxN];
static double h_W[2 * (kMaxN + 1)], h_sinp[kMaxN + 1], h_Bhat[2 * (kMaxN + 1)], h_dense[2 * (kMaxN + 1)];
static int h_pin[kMaxN + 1], h_pout[kMaxN + 1];

struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int n = 0;                      // (n, kappa) whose tables are on the device, n = 0: none
  double kappa = 0.0;
  DstPlan plan{};
};
constexpr int kMaxDevices = 64;
static DeviceState g_dev[kMaxDevices];
static std::mutex g_mutex;

// Build the tables of (n, kappa) in the host staging arrays and copy them into
// the table region of the device array; fills st.plan.  Synchronises `stream`.
cudaError_t upload_tables(DeviceState& st, int n, double kappa, cudaStream_t stream) {
  const int p = n + 1;
  const double delta = (double)p * (double)p;
  DstPlan dp{};
  dp.n = n;
  dp.p = p;
  // the plan and tables come from the library's host-table helpers (the same
  // functions the domain API uses), in their heap-free forms
  const HostPlan shape = plan_shape(n);
  dp.mode = shape.mode;
  dp.N = shape.N;
  dp.nrad = shape.nrad;
  for (int i = 0; i < shape.nrad; ++i) dp.rad[i] = shape.rad[i];
  const int N = dp.N;
  for (int j = 0; j < p; ++j) h_sinp[j] = cos_pi_frac(2 * j - p, 2 * p);  // sin(pi j/p)
  for (int m = 0; m < 2 * p; ++m) h_dense[m] = cos_pi_frac(2 * m - p, 2 * p);
  for (int m = 0; m < N; ++m) cexp_neg(m, N, &h_W[2 * m], &h_W[2 * m + 1]);
  if (dp.mode == DST_RADER) rader_tables(p, h_pin, h_pout, h_Bhat);
  fill_pivots_into(n, n, delta, kappa, h_rpiv);
  for (long long i = 0; i < (long long)n * n; ++i) h_mneg[i] = -delta * h_rpiv[i];

  // table region, after the coefficient area; 256-byte aligned pieces
  unsigned char* t = st.base + (size_t)kCoeffDoubles * 8;
  auto take = [&](size_t bytes) {
    unsigned char* q = t;
    t += (bytes + 255) & ~(size_t)255;
    return q;
  };
  double* rpiv = (double*)take(sizeof(double) * n * n);
  double* mneg = (double*)take(sizeof(double) * n * n);
  double* W = (double*)take(sizeof(double) * 2 * N);
  double* sinp = (double*)take(sizeof(double) * p);
  double* Bhat = (double*)take(sizeof(double) * 2 * N);
  double* dense = (double*)take(sizeof(double) * 2 * p);
  int* pin = (int*)take(sizeof(int) * N);
  int* pout = (int*)take(sizeof(int) * N);
  cudaError_t err = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (err == cudaSuccess) err = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
  };
  cp(rpiv, h_rpiv, sizeof(double) * n * n);
  cp(mneg, h_mneg, sizeof(double) * n * n);
  cp(W, h_W, sizeof(double) * 2 * N);
  cp(sinp, h_sinp, sizeof(double) * p);
  cp(dense, h_dense, sizeof(double) * 2 * p);
  if (dp.mode == DST_RADER) {
    cp(Bhat, h_Bhat, sizeof(double) * 2 * N);
    cp(pin, h_pin, sizeof(int) * N);
    cp(pout, h_pout, sizeof(int) * N);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);  // the staging arrays are reused
  if (err != cudaSuccess) return err;
  dp.W = W;
  dp.sinp = sinp;
  dp.Bhat = dp.mode == DST_RADER ? Bhat : nullptr;
  dp.dense = dense;
  dp.pin = dp.mode == DST_RADER ? pin : nullptr;
  dp.pout = dp.mode == DST_RADER ? pout : nullptr;
  st.plan = dp;
  st.n = n;
  st.kappa = kappa;
  return cudaSuccess;
}

}  // namespace

extern "C" fpg_status fpg_fast_solve_noalloc(int32_t n, double kappa, const double* v_dev, double* z_dev,
                                             int32_t nvec, void* stream) {
  if (!v_dev || !z_dev || nvec < 1) {
    record_message("fpg_fast_solve_noalloc: null pointer or nvec < 1");
    return FPG_EINVAL;
  }
  if (n < 2 || n > kMaxN) {
    record_message("fpg_fast_solve_noalloc: n outside 2..FPG_NOALLOC_MAX_N");
    return FPG_EINVAL;
  }
  if (!(kappa <= 0.0) || !std::isfinite(kappa)) {
    record_message("fpg_fast_solve_noalloc: kappa must be finite and <= 0");
    return FPG_EINVAL;
  }
  if (nvec > FPG_NOALLOC_MAX_NVEC) {
    // the batch is a grid dimension of the fast-solve launches; the cap matches
    // the domain API's largest right-hand-side count
    record_message("fpg_fast_solve_noalloc: nvec exceeds FPG_NOALLOC_MAX_NVEC");
    return FPG_EINVAL;
  }
  if ((long long)nvec * n * n > kCoeffDoubles) {
    record_message("fpg_fast_solve_noalloc: nvec * n * n exceeds FPG_NOALLOC_MAX_POINTS");
    return FPG_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  FPG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FPG_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& ds = g_dev[dev];
  if (!ds.ready) {
    // one-time set-up on this device, with this device current
    void* ptr = nullptr;
    FPG_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    ds.base = (unsigned char*)ptr;
    ds.ready = true;
  }
  if (ds.n != n || ds.kappa != kappa) {
    ds.n = 0;
    FPG_CUDA_TRY(upload_tables(ds, n, kappa, st));
  }
  unsigned char* t = ds.base + (size_t)kCoeffDoubles * 8;
  const size_t piv_bytes = ((sizeof(double) * (size_t)n * n + 255) & ~(size_t)255);
  FastSolveTables tb{};
  tb.n = n;
  tb.ns = n;
  tb.delta = (double)(n + 1) * (double)(n + 1);
  tb.plan = ds.plan;
  tb.rpiv = t;
  tb.mneg = t + piv_bytes;
  const LineLayout LC{n, n, 1, n};
  const BatchDesc bd{(long long)n * n, {0, 0, 0, 0}, 1};
  FPG_CUDA_TRY(launch_fast_solve(64, 64, tb, LC, v_dev, bd, z_dev, bd, nvec, ds.base, nullptr, 1, st, nullptr));
  return FPG_OK;
}
