// Standalone fast solves: rectangle plans for the three line transforms of
// Sec. 2.1-2.2 (DST-I Dirichlet, DCT-II Neumann, real-DFT periodic lines, each
// followed by one Thomas solve per mode and the inverse transform), their
// one-call forms for Neumann and periodic rectangles, and the 3-D box plan (the
// 3-D extension named after Sec. 2.1: DST-I along x and y, Thomas along z).
// Plans carve their FP64 tables and scratch from the caller's workspace once.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fpg_host_tables.h"
#include "fpg_internal.cuh"

namespace fpg {

cudaError_t launch_fast_solve(int prec, int out_prec, const FastSolveTables& tb, LineLayout L, const double* in,
                              BatchDesc ib, void* out, BatchDesc ob, int nblk, void* scratch, const int* active,
                              int nper_active, cudaStream_t st, int* launches, cudaEvent_t* ev = nullptr);
cudaError_t launch_dst_pass(bool forward, const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib,
                            double* scratch, double* out, BatchDesc ob, int nblk, cudaStream_t st);
cudaError_t launch_thomas_any(int prec, void* scratch, int n, int ns, const void* rpiv, const void* mneg, int nblk,
                              const int* active, int nper_active, cudaStream_t st, int wpb);
bool dct_plan_shape(int n, DstPlan* pl);
bool rdft_plan_shape(int n, DstPlan* pl);

}  // namespace fpg

using namespace fpg;

namespace {

fpg_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    record_cuda_error(e, "kernel launch");
    return FPG_ECUDA;
  }
  return FPG_OK;
}

}  // namespace

// ---- rectangle fast-solve plans (Sec. 2.1-2.2) --------------------------------
struct fpg_rect_plan {
  int kind = 0, nt = 0, ns = 0, nvec = 0;
  cudaStream_t st = nullptr;
  FastSolveTables tb;
  double* scratch = nullptr;
};

// ---- 3-D box fast-solve plans (the 3-D extension after Sec. 2.1) -------------
struct fpg_box_plan {
  int nx = 0, ny = 0, nz = 0, nvec = 0;
  cudaStream_t st = nullptr;
  FastSolveTables tx, ty;  // DST-I along x and along y (FP64)
  const void* rpiv = nullptr;  // Thomas along z per (kx, ky): [kx][ky][z]
  const void* mneg = nullptr;
  double *s1 = nullptr, *s2 = nullptr;  // [b][kx][y + ny z] and [b][kx][ky][z]
};

namespace {

// DST-I plan of length n with its FP64 tables carved from c (no copies).
DstPlan carve_dst_plan(int n, const HostPlan& hp, Carver& c) {
  DstPlan dp{};
  const int N = hp.N, pp = n + 1;
  dp.n = n; dp.p = pp; dp.mode = hp.mode; dp.N = N; dp.nrad = hp.nrad;
  for (int i = 0; i < kMaxRadices; ++i) dp.rad[i] = hp.rad[i];
  dp.W = c.take(sizeof(double) * 2 * N);
  dp.sinp = c.take(sizeof(double) * pp);
  dp.Bhat = hp.mode == DST_RADER ? c.take(sizeof(double) * 2 * N) : nullptr;
  dp.dense = c.take(sizeof(double) * 2 * pp);
  dp.pin = hp.mode == DST_RADER ? (const int*)c.take(sizeof(int) * N) : nullptr;
  dp.pout = hp.mode == DST_RADER ? (const int*)c.take(sizeof(int) * N) : nullptr;
  return dp;
}

cudaError_t copy_dst_plan(const DstPlan& pl, const HostPlan& hp, cudaStream_t st) {
  auto cp = [&](const void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(const_cast<void*>(dst), src, b, cudaMemcpyHostToDevice, st);
  };
  cudaError_t err = cp(pl.W, hp.W.data(), sizeof(double) * hp.W.size());
  if (!err) err = cp(pl.sinp, hp.sinp.data(), sizeof(double) * hp.sinp.size());
  if (!err) err = cp(pl.dense, hp.dense.data(), sizeof(double) * hp.dense.size());
  if (hp.mode == DST_RADER) {
    if (!err) err = cp(pl.Bhat, hp.Bhat.data(), sizeof(double) * hp.Bhat.size());
    if (!err) err = cp(pl.pin, hp.pin.data(), sizeof(int) * hp.pin.size());
    if (!err) err = cp(pl.pout, hp.pout.data(), sizeof(int) * hp.pout.size());
  }
  return err;
}

fpg_status box_validate(int32_t nx, int32_t ny, int32_t nz, int32_t nvec) {
  if (nx < 2 || ny < 2 || nz < 1 || nvec < 1 || nx > 4096 || ny > 4096 || nz > 4096) return FPG_EINVAL;
  if ((long long)nvec * nx > 65535) return FPG_EINVAL;  // the y pass runs one grid row per (vector, kx)
  return FPG_OK;
}

void box_carve(fpg_box_plan* R, int nx, int ny, int nz, int nvec, const HostPlan& hx, const HostPlan& hy,
               Carver& c) {
  const DstPlan px = carve_dst_plan(nx, hx, c);
  const DstPlan py = carve_dst_plan(ny, hy, c);
  const size_t pts = (size_t)nx * ny * nz;
  const void* r = c.take(sizeof(double) * pts);
  const void* m = c.take(sizeof(double) * pts);
  void* s1 = c.take(sizeof(double) * pts * nvec);
  void* s2 = c.take(sizeof(double) * pts * nvec);
  if (R) {
    R->tx.plan = px;
    R->ty.plan = py;
    R->rpiv = r;
    R->mneg = m;
    R->s1 = (double*)s1;
    R->s2 = (double*)s2;
  }
}

fpg_status rect_validate(int32_t kind, int32_t nt, int32_t ns, int32_t nvec) {
  if (nt < 2 || ns < 1 || nvec < 1 || ns > 4096) return FPG_EINVAL;
  DstPlan dp;
  switch (kind) {
    case FPG_RECT_DIRICHLET: return nt <= 4096 ? FPG_OK : FPG_EINVAL;
    case FPG_RECT_NEUMANN:
      if (nt > 2048 || (nt & 1)) return FPG_EINVAL;
      return dct_plan_shape(nt, &dp) ? FPG_OK : FPG_EUNSUPPORTED;
    case FPG_RECT_PERIODIC:
      if (nt > 2048) return FPG_EINVAL;
      return rdft_plan_shape(nt, &dp) ? FPG_OK : FPG_EUNSUPPORTED;
    default: return FPG_EINVAL;
  }
}

// Carves the plan's tables and scratch; with R == nullptr only sizes are taken.
void rect_carve(fpg_rect_plan* R, int kind, int nt, int ns, int nvec, const HostPlan& hp, Carver& c) {
  DstPlan dp{};
  const void* post = nullptr;
  if (kind == FPG_RECT_DIRICHLET) {
    dp = carve_dst_plan(nt, hp, c);
  } else {
    if (kind == FPG_RECT_NEUMANN) dct_plan_shape(nt, &dp);
    else rdft_plan_shape(nt, &dp);
    dp.W = c.take(sizeof(double) * 2 * nt);
    post = c.take(sizeof(double) * 2 * nt);
  }
  const size_t pts = (size_t)nt * ns;
  const void* r = c.take(sizeof(double) * pts);
  const void* m = c.take(sizeof(double) * pts);
  void* s = c.take(sizeof(double) * pts * nvec);
  if (R) {
    R->tb.plan = dp;
    R->tb.post = post;
    R->tb.rpiv = r;
    R->tb.mneg = m;
    R->scratch = (double*)s;
  }
}

}  // namespace

extern "C" {

fpg_status fpg_rect_plan_bytes(int32_t kind, int32_t nt, int32_t ns, int32_t nvec, size_t* bytes) {
  if (!bytes) return FPG_EINVAL;
  FPG_TRY(rect_validate(kind, nt, ns, nvec));
  HostPlan hp = kind == FPG_RECT_DIRICHLET ? plan_shape(nt) : HostPlan{};
  Carver c(nullptr);
  rect_carve(nullptr, kind, nt, ns, nvec, hp, c);
  *bytes = c.used + 256;
  return FPG_OK;
}

fpg_status fpg_rect_plan_create(int32_t kind, int32_t nt, int32_t ns, double h, double kappa, int32_t nvec,
                                void* ws, size_t bytes, void* stream, fpg_rect_plan** out) {
  if (!out || !ws || !(h > 0.0) || !(kappa <= 0.0) || !std::isfinite(kappa)) return FPG_EINVAL;
  *out = nullptr;
  size_t need = 0;
  FPG_TRY(fpg_rect_plan_bytes(kind, nt, ns, nvec, &need));
  if (bytes < need) return FPG_ENOMEM;
  fpg_rect_plan* R = new (std::nothrow) fpg_rect_plan();
  if (!R) return FPG_ENOMEM;
  R->kind = kind;
  R->nt = nt;
  R->ns = ns;
  R->nvec = nvec;
  R->st = (cudaStream_t)stream;
  const double delta = 1.0 / (h * h);
  R->tb.n = nt;
  R->tb.ns = ns;
  R->tb.delta = delta;
  R->tb.kind = kind == FPG_RECT_DIRICHLET ? 0 : (kind == FPG_RECT_NEUMANN ? 1 : 2);
  HostPlan hp = kind == FPG_RECT_DIRICHLET ? build_plan(nt) : HostPlan{};
  Carver c(ws);
  rect_carve(R, kind, nt, ns, nvec, hp, c);
  std::vector<double> r, m, W, post;
  if (kind == FPG_RECT_DIRICHLET) {
    fill_pivots(nt, ns, delta, kappa, r);
    m.resize(r.size());
    for (size_t i = 0; i < r.size(); ++i) m[i] = -delta * r[i];
  } else {
    dct_tables(nt, W, post);
    if (kind == FPG_RECT_NEUMANN) dct_pivots(nt, ns, delta, kappa, 0.0, 0, r, m);
    else rdft_pivots(nt, ns, delta, kappa, r, m);
  }
  auto cp = [&](const void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(const_cast<void*>(dst), src, b, cudaMemcpyHostToDevice, R->st);
  };
  const DstPlan& pl = R->tb.plan;
  cudaError_t err = cp(R->tb.rpiv, r.data(), sizeof(double) * r.size());
  if (!err) err = cp(R->tb.mneg, m.data(), sizeof(double) * m.size());
  if (kind == FPG_RECT_DIRICHLET) {
    if (!err) err = copy_dst_plan(pl, hp, R->st);
  } else {
    if (!err) err = cp(pl.W, W.data(), sizeof(double) * W.size());
    if (!err) err = cp(R->tb.post, post.data(), sizeof(double) * post.size());
  }
  // the host tables are freed on return: wait for the copies
  if (!err) err = cudaStreamSynchronize(R->st);
  if (err) {
    record_cuda_error(err, "fpg_rect_plan_create");
    delete R;
    return FPG_ECUDA;
  }
  *out = R;
  return FPG_OK;
}

fpg_status fpg_rect_solve(fpg_rect_plan* R, const double* v, double* z, int32_t nvec) {
  if (!R || !v || !z || nvec < 0 || nvec > R->nvec) return FPG_EINVAL;
  const LineLayout L{R->nt, R->ns, 1, R->nt};
  const BatchDesc bd{(long long)R->nt * R->ns, {0, 0, 0, 0}, 1};
  int nl = 0;
  FPG_CUDA_TRY(launch_fast_solve(64, 64, R->tb, L, v, bd, z, bd, nvec, R->scratch, nullptr, 1, R->st, &nl));
  return check_launch();
}

void fpg_rect_plan_destroy(fpg_rect_plan* R) { delete R; }

// One-call forms for the Neumann and periodic rectangles: plan, solve, release.
fpg_status fpg_neumann_workspace_bytes(int32_t nt, int32_t ns, int32_t nvec, size_t* bytes) {
  return fpg_rect_plan_bytes(FPG_RECT_NEUMANN, nt, ns, nvec, bytes);
}

fpg_status fpg_periodic_workspace_bytes(int32_t nt, int32_t ns, int32_t nvec, size_t* bytes) {
  return fpg_rect_plan_bytes(FPG_RECT_PERIODIC, nt, ns, nvec, bytes);
}

static fpg_status rect_once(int32_t kind, int32_t nt, int32_t ns, double h, double kappa, const double* v, double* z,
                     int32_t nvec, void* ws, size_t bytes, void* stream) {
  if (!v || !z) return FPG_EINVAL;
  fpg_rect_plan* R = nullptr;
  FPG_TRY(fpg_rect_plan_create(kind, nt, ns, h, kappa, nvec, ws, bytes, stream, &R));
  const fpg_status s = fpg_rect_solve(R, v, z, nvec);
  fpg_rect_plan_destroy(R);
  return s;
}

fpg_status fpg_neumann_solve(int32_t nt, int32_t ns, double h, double kappa, const double* v, double* z, int32_t nvec,
                             void* ws, size_t bytes, void* stream) {
  return rect_once(FPG_RECT_NEUMANN, nt, ns, h, kappa, v, z, nvec, ws, bytes, stream);
}

fpg_status fpg_periodic_solve(int32_t nt, int32_t ns, double h, double kappa, const double* v, double* z,
                              int32_t nvec, void* ws, size_t bytes, void* stream) {
  return rect_once(FPG_RECT_PERIODIC, nt, ns, h, kappa, v, z, nvec, ws, bytes, stream);
}

fpg_status fpg_box_plan_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t nvec, size_t* bytes) {
  if (!bytes) return FPG_EINVAL;
  FPG_TRY(box_validate(nx, ny, nz, nvec));
  Carver c(nullptr);
  box_carve(nullptr, nx, ny, nz, nvec, plan_shape(nx), plan_shape(ny), c);
  *bytes = c.used + 256;
  return FPG_OK;
}

fpg_status fpg_box_plan_create(int32_t nx, int32_t ny, int32_t nz, double h, double kappa, int32_t nvec, void* ws,
                               size_t bytes, void* stream, fpg_box_plan** out) {
  if (!out || !ws || !(h > 0.0) || !(kappa <= 0.0) || !std::isfinite(kappa)) return FPG_EINVAL;
  *out = nullptr;
  size_t need = 0;
  FPG_TRY(fpg_box_plan_bytes(nx, ny, nz, nvec, &need));
  if (bytes < need) return FPG_ENOMEM;
  fpg_box_plan* R = new (std::nothrow) fpg_box_plan();
  if (!R) return FPG_ENOMEM;
  R->nx = nx;
  R->ny = ny;
  R->nz = nz;
  R->nvec = nvec;
  R->st = (cudaStream_t)stream;
  const double delta = 1.0 / (h * h);
  HostPlan hx = build_plan(nx), hy = build_plan(ny);
  Carver c(ws);
  box_carve(R, nx, ny, nz, nvec, hx, hy, c);
  R->tx.n = nx;
  R->tx.ns = ny * nz;
  R->ty.n = ny;
  R->ty.ns = nz;
  R->tx.delta = R->ty.delta = delta;
  // Thomas along z for mode (kx, ky): diagonal -6 delta + 2 delta cos(kx pi/(nx+1))
  // + 2 delta cos(ky pi/(ny+1)) + kappa, off-diagonals delta
  std::vector<double> r((size_t)nx * ny * nz), m(r.size());
  for (int kx = 1; kx <= nx; ++kx)
    for (int ky = 1; ky <= ny; ++ky) {
      const double d = -6.0 * delta + 2.0 * delta * cos_pi_frac(kx, nx + 1) + 2.0 * delta * cos_pi_frac(ky, ny + 1) +
                       kappa;
      const size_t o = ((size_t)(kx - 1) * ny + (ky - 1)) * nz;
      double rp = 0.0;
      for (int s = 0; s < nz; ++s) {
        rp = s == 0 ? 1.0 / d : 1.0 / (d - delta * delta * rp);
        r[o + s] = rp;
        m[o + s] = -delta * rp;
      }
    }
  cudaError_t err = copy_dst_plan(R->tx.plan, hx, R->st);
  if (!err) err = copy_dst_plan(R->ty.plan, hy, R->st);
  if (!err) err = cudaMemcpyAsync(const_cast<void*>(R->rpiv), r.data(), sizeof(double) * r.size(),
                                  cudaMemcpyHostToDevice, R->st);
  if (!err) err = cudaMemcpyAsync(const_cast<void*>(R->mneg), m.data(), sizeof(double) * m.size(),
                                  cudaMemcpyHostToDevice, R->st);
  if (!err) err = cudaStreamSynchronize(R->st);  // the host tables are freed on return
  if (err) {
    record_cuda_error(err, "fpg_box_plan_create");
    delete R;
    return FPG_ECUDA;
  }
  *out = R;
  return FPG_OK;
}

fpg_status fpg_box_solve(fpg_box_plan* R, const double* v, double* z, int32_t nvec) {
  if (!R || !v || !z || nvec < 0 || nvec > R->nvec) return FPG_EINVAL;
  if (nvec == 0) return FPG_OK;
  const int nx = R->nx, ny = R->ny, nz = R->nz;
  const long long pts = (long long)nx * ny * nz, plane = (long long)ny * nz;
  const LineLayout Lx{nx, ny * nz, 1, nx};  // lines along x, s = y + ny z
  const LineLayout Ly{ny, nz, 1, ny};       // lines along y inside one (vector, kx) slab, s = z
  const BatchDesc bx{pts, {0, 0, 0, 0}, 1};
  const BatchDesc by{plane, {0, 0, 0, 0}, 1};
  const BatchDesc none{0, {0, 0, 0, 0}, 1};
  FPG_CUDA_TRY(launch_dst_pass(true, R->tx, Lx, v, bx, R->s1, nullptr, none, nvec, R->st));
  FPG_CUDA_TRY(launch_dst_pass(true, R->ty, Ly, R->s1, by, R->s2, nullptr, none, nvec * nx, R->st));
  FPG_CUDA_TRY(launch_thomas_any(64, R->s2, nx * ny, nz, R->rpiv, R->mneg, nvec, nullptr, 1, R->st, 0));
  FPG_CUDA_TRY(launch_dst_pass(false, R->ty, Ly, nullptr, none, R->s2, R->s1, by, nvec * nx, R->st));
  FPG_CUDA_TRY(launch_dst_pass(false, R->tx, Lx, nullptr, none, R->s1, z, bx, nvec, R->st));
  return check_launch();
}

void fpg_box_plan_destroy(fpg_box_plan* R) { delete R; }

}  // extern "C"
