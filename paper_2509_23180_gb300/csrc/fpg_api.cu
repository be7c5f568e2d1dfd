// C ABI of the solver (include/fpg.h): domain set-up, workspace carving, host
// tables in FP64, the flexible-GMRES driver of Alg. "fft_dd_solver", and the
// per-step operator entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fpg_host_tables.h"
#include "fpg_internal.cuh"
#include "fpg_lattice_host.h"

namespace fpg {

cudaError_t launch_fast_solve(int prec, int out_prec, const FastSolveTables& tb, LineLayout L, const double* in,
                              BatchDesc ib, void* out, BatchDesc ob, int nblk, void* scratch, const int* active,
                              int nper_active, cudaStream_t st, int* launches, cudaEvent_t* ev = nullptr);
bool schur_dst_supported(int n);
cudaError_t launch_schur_dst(const void* z, int zprec, long long zstride, int n, const DstPlan& pl, const double* gsc,
                             const int* arms, int narms, double* corr, const int* active, int nrhs, cudaStream_t st);
cudaError_t launch_schur_gmat(const void* z, int zprec, long long zstride, int n, const double* G, const int* arms_dev,
                              int narms, double* corr, const int* active, int nrhs, cudaStream_t st);
cudaError_t launch_schur_reduced(const void* z, int zprec, long long zstride, int n, const double* ctab,
                                 const int* arms_dev, int narms, double* corr, const int* active, int nrhs,
                                 cudaStream_t st);
cudaError_t launch_stencil_c(const void* z, int zprec, long long zstride, double* w, long long wstride, int n,
                             double delta, double kappa, const double* corr, int armmask, const int* active,
                             int nrhs, int gx, cudaStream_t st);
cudaError_t launch_literal_inject(const void* z, int zprec, long long zstride, int n, double delta,
                                  double* armbuf, long long rhs_stride, ArmOffsets ao, const int* active,
                                  int nrhs, int gx, cudaStream_t st);
cudaError_t launch_literal_extract(const double* armsol, long long rhs_stride, ArmOffsets ao, int n,
                                   double delta, double* corr, const int* active, int nrhs, cudaStream_t st);
cudaError_t launch_mgs(const double* V, long long vstride, double* w, double* vout, long long len, int j,
                       int nrhs, double* part, int gmax, double* H, int hcol_stride, int hrhs_stride,
                       const int* active, int gx, cudaStream_t st, int* launches);
cudaError_t launch_givens(double* H, int hcol_stride, int hrhs_stride, double* cs, double* sn, double* g,
                          double* res, int j, int m, int nrhs, const double* tolabs, int* active, int* kcyc,
                          int* iters, int max_iters, cudaStream_t st);
cudaError_t launch_cycle_end(const double* H, int hcol_stride, int hrhs_stride, const double* g, double* y,
                             int m, int nrhs, const int* kcyc, double* u, const void* Z, int zprec,
                             long long zvstride, long long len, int gx, cudaStream_t st);
cudaError_t launch_restart(const double* fc, const double* w, double* v0, long long len, int nrhs, double* part,
                           int gmax, double* g, int m, const double* tolabs, double* rnorm, int* done,
                           int* active, int* kcyc, const int* iters, int max_iters, int gx, cudaStream_t st);
cudaError_t launch_reduce_rhs(const double* f, const double* q, long long ntot, int n, double delta,
                              ArmOffsets ao, double* fc, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_arm_rhs(const double* f, const double* u, long long ntot, int n, double delta, ArmOffsets ao,
                           double* out, double* p, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_global_apply(const double* p, double* y, const double* f, long long ntot, int n, double delta,
                                double kappa, ArmOffsets ao, double* part, int gmax, int nrhs, int gx,
                                double* rel_out, double* fnorm_out, double rtol, double* tolabs,
                                cudaStream_t st);
cudaError_t launch_fma_probe(int prec, int blocks, int iters, cudaStream_t st);
cudaError_t launch_refine_rhs(const double* f, double* r, const double* gres, double rtol, long long ntot, int nrhs,
                              int* resume_count, int gx, cudaStream_t st);
cudaError_t launch_add_vec(double* p, const double* q, long long total, cudaStream_t st);
cudaError_t launch_refine_tol(double* tolabs, const double* fnorm0, double scale, int nrhs, cudaStream_t st);
cudaError_t launch_precond_simple(const double* v, void* z, int zprec, long long len, int n, double delta,
                                  double kappa, const double* ctab, int armmask, int jacobi, const int* active,
                                  int nrhs, int gx, cudaStream_t st);
int arnoldi_cluster_size(long long len);
int fast_solve_path(int prec, const FastSolveTables& tb, LineLayout L, int nblk);
bool dct_plan_shape(int n, DstPlan* pl);
bool rdft_plan_shape(int n, DstPlan* pl);
cudaError_t launch_record_history(const double* res, const int* iters, double* hist, int len, int nrhs,
                                  cudaStream_t st);
cudaError_t launch_chain_schur(const void* z, int zprec, long long zstride, const ChainGeom& G, const double* ctab,
                               double* corr, const int* active, int nrhs, cudaStream_t st);
cudaError_t launch_chain_stencil(const void* z, int zprec, long long zstride, double* w, long long wstride,
                                 const ChainGeom& G, double delta, double kappa, const double* corr,
                                 const int* active, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_chain_reduce_rhs(const double* f, const double* q, long long ntot, const ChainGeom& G,
                                    double delta, double* fc, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_chain_arm_rhs(const double* f, const double* u, long long ntot, const ChainGeom& G, double delta,
                                 double* out, double* p, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_chain_global_apply(const double* p, double* y, const double* f, long long ntot, const ChainGeom& G,
                                      double delta, double kappa, double* part, int gmax, int nrhs, int gx,
                                      double* rel_out, double* fnorm_out, double rtol, double* tolabs,
                                      cudaStream_t st);
cudaError_t launch_dst_pass(bool forward, const FastSolveTables& tb, LineLayout L, const double* in, BatchDesc ib,
                            double* scratch, double* out, BatchDesc ob, int nblk, cudaStream_t st);
cudaError_t launch_thomas_any(int prec, void* scratch, int n, int ns, const void* rpiv, const void* mneg, int nblk,
                              const int* active, int nper_active, cudaStream_t st, int wpb);
int arnoldi_reg_ept(long long len, int csz, int ntcap);
int arnoldi_reg_threads(long long len, int csz, int ept);
cudaError_t launch_arnoldi_reg(int csz, int ntcap, const double* V, long long vstride, const double* w,
                               const void* z, int zprec, const double* corr, int n, double delta, double kappa, int armmask,
                               double* vout, long long len, int j, int nrhs, double* H, int hcol_stride,
                               int hrhs_stride, double* cs, double* sn, double* g, double* res, int m,
                               const double* tolabs, int* active, int* kcyc, int* iters, int max_iters, int do_givens,
                               int* err, cudaStream_t st);
cudaError_t launch_arnoldi_cluster(int csz, const double* V, long long vstride, double* w, double* vout,
                                   long long len, int j, int nrhs, double* H, int hcol_stride, int hrhs_stride,
                                   double* cs, double* sn, double* g, double* res, int m, const double* tolabs,
                                   int* active, int* kcyc, int* iters, int max_iters, int do_givens,
                                   cudaStream_t st);
cudaError_t launch_arm_residual(const double* rhs, const double* x, double* out, long long ntot, int n, double delta,
                                double kappa, ArmOffsets ao, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_arm_add(double* x, const double* e, long long ntot, int n, ArmOffsets ao, int nrhs, int gx,
                           cudaStream_t st);

static thread_local char g_last_err[256] = "no error";

void record_cuda_error(cudaError_t e, const char* where) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s", cudaGetErrorString(e), where);
}

void record_message(const char* msg) { snprintf(g_last_err, sizeof(g_last_err), "%s", msg); }

}  // namespace fpg

using namespace fpg;

namespace {

constexpr int kGmax = 1024;
constexpr int kPhases = 11;  // 7..9: the three fast-solve kernels of a1; 10: the fused one-pass kernel
constexpr int kMaxEvents = 8192;
// The Schur iteration stops at this fraction of the requested relative residual,
// so that the global residual (which adds the rounding of the arm back
// substitution) still meets the request.
constexpr double kInnerMargin = 0.9;
// Acceptance checks per solve: after back substitution a right-hand side above
// rtol resumes with its Schur target scaled by 1/4, at most this many times.
constexpr int kAcceptRounds = 3;


struct Layout {
  int n, narms, armmask;
  long long nc, na, ntot;
  ArmOffsets ao;
  int arm_slots[4];
  int chain = 0;  // K of a chain of crosses (0: L, T or cross)
  ChainGeom cg;   // the chain's row width and arm offsets
  int lattice = 0;  // 1: general concatenated geometry (FPG_GEOM_LATTICE)
  LatticeGeom lg;
  // the arm kernels (residual, update) take up to four arms, slots W, E (n+1 wide)
  // and S, N (n+1 tall); the arms of a chain or a lattice go in several groups
  std::vector<ArmOffsets> arm_groups;
};

bool make_layout(const fpg_domain_desc* d, Layout* L) {
  const int n = d->n;
  const int as = d->boundary == FPG_BC_NEUMANN_SIDES ? n : n + 1;
  L->n = n;
  L->nc = (long long)n * n;
  L->na = (long long)n * as;
  L->ao.as = as;
  L->ao.bc = d->boundary == FPG_BC_NEUMANN_SIDES ? 1 : 0;
  L->arm_groups.clear();
  if (d->geometry == FPG_GEOM_LATTICE) {
    if (!lattice_shape(d->lattice, n, &L->lg)) return false;
    const LatticeGeom& g = L->lg;
    L->lattice = 1;
    L->nc = g.nc;
    L->ntot = g.ntot;
    L->narms = g.nfaces;
    L->armmask = 0;
    for (int i = 0; i < 4; ++i) L->arm_slots[i] = i;
    const int groups = (std::max(g.nwe, g.nsn) + 1) / 2;
    for (int k = 0; k < groups; ++k) {
      ArmOffsets ao = L->ao;
      ao.off[0] = 2 * k < g.nwe ? g.we_off[2 * k] : -1;
      ao.off[1] = 2 * k + 1 < g.nwe ? g.we_off[2 * k + 1] : -1;
      ao.off[2] = 2 * k < g.nsn ? g.sn_off[2 * k] : -1;
      ao.off[3] = 2 * k + 1 < g.nsn ? g.sn_off[2 * k + 1] : -1;
      L->arm_groups.push_back(ao);
    }
    if (L->arm_groups.empty()) {
      for (int a = 0; a < 4; ++a) L->ao.off[a] = -1;
    } else {
      L->ao = L->arm_groups[0];
    }
    return true;
  }
  if (d->geometry == FPG_GEOM_CHAIN) {
    const int K = d->chain;
    L->chain = K;
    L->cg.K = K;
    L->cg.n = n;
    L->cg.nxc = (2 * K - 1) * (n + 1) - 1;
    L->nc = (long long)L->cg.nxc * n;
    L->narms = 2 * K + 2;
    L->armmask = 0;
    for (int s = 0; s < L->narms; ++s) L->cg.off[s] = L->nc + (long long)s * L->na;
    // ao: the first group (W, E, S_1, N_1) for the arm kernels; the rest go group by group
    L->ao.off[0] = L->cg.off[0];
    L->ao.off[1] = L->cg.off[1];
    L->ao.off[2] = L->cg.off[2];
    L->ao.off[3] = L->cg.off[2 + K];
    for (int i = 0; i < 4; ++i) L->arm_slots[i] = i;
    L->ntot = L->nc + (long long)L->narms * L->na;
    for (int g = 0; g < K; ++g) {  // (W, E, S_1, N_1), (-, -, S_2, N_2), ...
      ArmOffsets ao = L->ao;
      if (g > 0) ao.off[0] = ao.off[1] = -1, ao.off[2] = L->cg.off[2 + g], ao.off[3] = L->cg.off[2 + K + g];
      L->arm_groups.push_back(ao);
    }
    return true;
  }
  static const int slots_cross[] = {0, 1, 2, 3};
  static const int slots_t[] = {0, 1, 2};
  static const int slots_l[] = {1, 3};
  const int* slots;
  int cnt;
  switch (d->geometry) {
    case FPG_GEOM_CROSS: slots = slots_cross; cnt = 4; break;
    case FPG_GEOM_T: slots = slots_t; cnt = 3; break;
    case FPG_GEOM_L: slots = slots_l; cnt = 2; break;
    default: return false;
  }
  L->narms = cnt;
  L->armmask = 0;
  for (int a = 0; a < 4; ++a) L->ao.off[a] = -1;
  long long off = L->nc;
  for (int i = 0; i < cnt; ++i) {
    L->arm_slots[i] = slots[i];
    L->ao.off[slots[i]] = off;
    L->armmask |= 1 << slots[i];
    off += L->na;
  }
  L->ntot = off;
  L->arm_groups.push_back(L->ao);
  return true;
}

fpg_status validate(const fpg_domain_desc* d) {
  if (!d) return FPG_EINVAL;
  if (d->geometry < 0 || d->geometry > 4) return FPG_EINVAL;
  if (d->geometry == FPG_GEOM_LATTICE) {
    LatticeGeom g;
    if (d->chain != 0 || d->n < 2 || d->n > 4096 || !lattice_shape(d->lattice, d->n, &g)) return FPG_EINVAL;
    if (g.nwe > 8 || g.nsn > 8) return FPG_EUNSUPPORTED;  // one batch of the arm kernels per shape
    if (d->boundary != FPG_BC_DIRICHLET || d->schur_mode != FPG_SCHUR_REDUCED) return FPG_EUNSUPPORTED;
    if (g.ntot > (1LL << 31) - 1) return FPG_EUNSUPPORTED;  // 32-bit neighbour tables
  } else if (d->lattice != 0) {
    return FPG_EINVAL;
  }
  if (d->geometry == FPG_GEOM_CHAIN) {
    if (d->chain < 2 || d->chain > 5) return FPG_EINVAL;
    if (d->boundary != FPG_BC_DIRICHLET || d->schur_mode != FPG_SCHUR_REDUCED) return FPG_EUNSUPPORTED;
  } else if (d->chain != 0) {
    return FPG_EINVAL;
  }
  if (d->n < 2 || d->n > 4096) return FPG_EINVAL;
  if (!(d->kappa <= 0.0) || !std::isfinite(d->kappa)) return FPG_EINVAL;
  if (d->nrhs < 1 || d->nrhs > 4096) return FPG_EINVAL;
  if (d->restart < 1 || d->restart > 128) return FPG_EINVAL;
  if (!(d->rtol > 0.0) || !(d->rtol < 1.0)) return FPG_EINVAL;
  if (d->max_iters < 1) return FPG_EINVAL;
  if (d->precond_precision != 64 && d->precond_precision != 32) return FPG_EINVAL;
  if (d->schur_mode != FPG_SCHUR_REDUCED && d->schur_mode != FPG_SCHUR_LITERAL) return FPG_EINVAL;
  if (d->boundary != FPG_BC_DIRICHLET && d->boundary != FPG_BC_NEUMANN_SIDES) return FPG_EINVAL;
  if (d->boundary == FPG_BC_NEUMANN_SIDES) {
    // the arms' DCT-II lines: cross only, n even with prime factors <= 13, n <= 2048
    DstPlan dp;
    if (d->geometry != FPG_GEOM_CROSS || !dct_plan_shape(d->n, &dp)) return FPG_EUNSUPPORTED;
  }
  return FPG_OK;
}

int pick_gx(long long len, int nrhs) {
  long long want = (4LL * 152 + nrhs - 1) / nrhs;
  long long cap = (len + 255) / 256;
  long long g = std::min(want, cap);
  g = std::max(1LL, std::min(g, (long long)kGmax));
  return (int)g;
}

}  // namespace

struct fpg_domain {
  fpg_domain_desc desc;
  Layout L;
  cudaStream_t st;
  double delta;
  int prec;
  LineLayout LC, LWE, LSN;
  BatchDesc we, sn;  // arm groups inside full vectors
  BatchDesc sn2;     // chain: the N arms (sn holds the S arms)
  BatchDesc cb1, cb2;      // chain: the row's squares with n + 1 columns, and the last square
  LineLayout LC1, LC2;     // chain: their line layouts (transform along y, sweep along x)
  FastSolveTables tC64, tC32, tA64, tA32;
  FastSolveTables tA64e;  // Neumann-sided arms whose far end is row ns-1 (E, N); tA64 serves W, S
  FastSolveTables tR64, tR32;  // chain: the whole coupled row as one block (its A_c)
  LineLayout LR;
  double* ctab;
  double* gmat = nullptr;  // reduced Schur form: G(i, j) = T(|i-j|) - H(i+j), n x n (cross, T, L)
  double* gsc;           // [n] g_k delta^2 / (2 (n+1)), the transform form of the reduced Schur term
  int schur_transform = 0;  // 1: reduced Schur term by two DST-I per line where compiled (else the table sum)
  int arm_refine = 1;       // FP64 refinement steps of every arm solve (setup and finish)
  int* arms_dev;
  double *f, *tmp, *tmp2, *pbuf, *lit_in, *lit_out, *corr, *gres, *fnorm;
  double *rbuf, *psave, *fnorm0;  // global refinement: residual RHS, saved iterate, ||f||
  double* f_orig = nullptr;       // the caller's RHS while a refinement solve runs on rbuf
  bool refining = false;
  int* resume_dev = nullptr;
  int* err_dev = nullptr;   // status word of the bounded device waits (1: a wait gave up)
  LatticeDev lat;           // FPG_GEOM_LATTICE: neighbour, face and coupling tables
  void* scratch;
  KrylovState ks;
  int gx, gxf;
  // host mirrors
  std::vector<int> h_done, h_iters, h_kcyc;
  // measurement
  bool profiling = false;
  long long launches = 0;
  double phase_ms[kPhases] = {0};
  long long phase_launches[kPhases] = {0};
  std::vector<cudaEvent_t> evpool;
  std::vector<std::pair<int, int>> ev_used;  // (phase, event index of start)
  int ev_next = 0;
  int cycles_run = 0;
  bool use_cluster = true;
  int arnoldi_mode = 1;  // 1: register-resident fused kernel when it fits; 2: global-w cluster kernel
  int tune_csz = 0;      // Arnoldi cluster size chosen by fpg_autotune (0: built-in choice)
  int tune_nt = 0;       // thread cap per CTA of the register Arnoldi kernel (0: 256, else 512)
  bool use_graphs = true;
  int precond_kind = 0;  // 0: A_c^{-1} (the paper's), 1: identity, 2: Jacobi, 3: chain, block diagonal
  int accept_rounds = 0;  // acceptance checks done in the current solve
  cudaGraphExec_t cycle_exec = nullptr;
  long long cycle_kernels = 0;
  bool capturing = false;           // a restart cycle is being captured
  bool graph_profiled = false;      // the captured graph carries profiling events
  bool replay_pending = false;      // a profiled replay has not been read yet
  std::vector<cudaEvent_t> gev;     // events recorded by the graph
  std::vector<std::pair<int, int>> gev_used;
  int gev_next = 0;
  long long cycle_phase_launches[16] = {0};
  // staged solve
  bool first_cycle = true;
  double* p_cur = nullptr;
  int* h_done_pinned = nullptr;  // pinned host copy of the done flags
  cudaEvent_t ev_flags = nullptr;
  int bphase = 0;  // non-blocking staged solve: 0 idle, 1 restart issued, 2 finish issued
  double* hist = nullptr;  // caller's residual-history buffer [nrhs][hist_len] (fpg_set_history)
  int hist_len = 0;
};

namespace {

// The FP64 Thomas kernel's carry products, for each mode k and each chunk of
// thomas_chunk_rows(ns) rows: pf[k][s] = m_{c0} m_{c0+1} ... m_s (from the chunk's first
// row c0) and pb[k][s] = m_{c1} m_{c1-1} ... m_s (from its last row c1), multiplied in
// the kernel's own order so that the kernel's results do not change.
void thomas_chunk_products(int n, int ns, const std::vector<double>& m, std::vector<double>& pf,
                           std::vector<double>& pb) {
  pf.assign((size_t)n * ns, 0.0);
  pb.assign((size_t)n * ns, 0.0);
  const int C = thomas_chunk_rows(ns);
  if (C == 0) return;
  for (int k = 0; k < n; ++k) {
    const size_t row = (size_t)k * ns;
    for (int c0 = 0; c0 < ns; c0 += C) {
      const int c1 = std::min(ns, c0 + C) - 1;
      double q = 1.0;
      for (int s = c0; s <= c1; ++s) {
        q *= m[row + s];
        pf[row + s] = q;
      }
      q = 1.0;
      for (int s = c1; s >= c0; --s) {
        q *= m[row + s];
        pb[row + s] = q;
      }
    }
  }
}

// Carves every region; with base == nullptr only sizes are computed.
void carve(fpg_domain* D, const fpg_domain_desc* d, const Layout& L, const HostPlan* plan, Carver& c) {
  const int n = d->n, nrhs = d->nrhs, m = d->restart;
  const size_t zel = d->precond_precision == 64 ? 8 : 4;
  void* p;
  {
    const HostPlan& hp = *plan;
    const int N = hp.N, pp = n + 1;
    for (int prec = 64; prec >= 32; prec -= 32) {
      const size_t el = prec == 64 ? 8 : 4;
      DstPlan dp{};
      dp.n = n; dp.p = pp; dp.mode = hp.mode; dp.N = N; dp.nrad = hp.nrad;
      for (int i = 0; i < kMaxRadices; ++i) dp.rad[i] = hp.rad[i];
      dp.W = c.take(el * 2 * N);
      dp.sinp = c.take(el * pp);
      dp.Bhat = hp.mode == DST_RADER ? c.take(el * 2 * N) : nullptr;
      dp.dense = c.take(el * 2 * pp);
      dp.pin = hp.mode == DST_RADER ? (const int*)c.take(sizeof(int) * N) : nullptr;
      dp.pout = hp.mode == DST_RADER ? (const int*)c.take(sizeof(int) * N) : nullptr;
      if (D) {
        if (prec == 64) D->tC64.plan = D->tA64.plan = dp;
        else D->tC32.plan = D->tA32.plan = dp;
      }
    }
  }
  p = c.take(sizeof(double) * L.nc);          if (D) D->tC64.rpiv = p;
  p = c.take(sizeof(float) * L.nc);           if (D) D->tC32.rpiv = p;
  p = c.take(sizeof(double) * L.na);          if (D) D->tA64.rpiv = p;
  p = c.take(sizeof(float) * L.na);           if (D) D->tA32.rpiv = p;
  p = c.take(sizeof(double) * L.nc);          if (D) D->tC64.mneg = p;
  p = c.take(sizeof(float) * L.nc);           if (D) D->tC32.mneg = p;
  p = c.take(sizeof(double) * L.na);          if (D) D->tA64.mneg = p;
  p = c.take(sizeof(float) * L.na);           if (D) D->tA32.mneg = p;
  // FP64 Thomas: in-chunk products of mneg (centre, and Dirichlet arms)
  p = c.take(sizeof(double) * L.nc);          if (D) D->tC64.pfwd = p;
  p = c.take(sizeof(double) * L.nc);          if (D) D->tC64.pbwd = p;
  if (d->boundary != FPG_BC_NEUMANN_SIDES) {
    p = c.take(sizeof(double) * L.na);        if (D) D->tA64.pfwd = p;
    p = c.take(sizeof(double) * L.na);        if (D) D->tA64.pbwd = p;
  }
  if (d->boundary == FPG_BC_NEUMANN_SIDES) {
    // arms: DCT-II lines along t, pivots with the far-end row first (W, S) or last (E, N)
    DstPlan dp;
    dct_plan_shape(n, &dp);
    dp.W = c.take(sizeof(double) * 2 * n);
    const void* post = c.take(sizeof(double) * 2 * n);
    const void* r2 = c.take(sizeof(double) * L.na);
    const void* m2 = c.take(sizeof(double) * L.na);
    if (D) {
      for (FastSolveTables* tb : {&D->tA64, &D->tA64e}) {
        tb->plan = dp;
        tb->post = post;
        tb->kind = 1;
      }
      D->tA64e.rpiv = r2;
      D->tA64e.mneg = m2;
    }
  }
  if (L.chain) {  // the coupled row's own sweeps: n modes of nxc rows
    const size_t rows = (size_t)n * L.cg.nxc;
    p = c.take(sizeof(double) * rows); if (D) D->tR64.rpiv = p;
    p = c.take(sizeof(double) * rows); if (D) D->tR64.mneg = p;
    p = c.take(sizeof(float) * rows);  if (D) D->tR32.rpiv = p;
    p = c.take(sizeof(float) * rows);  if (D) D->tR32.mneg = p;
  }
  p = c.take(sizeof(double) * (4 * n + 2));   if (D) D->ctab = (double*)p;
  if (!L.chain && !L.lattice && d->schur_mode == FPG_SCHUR_REDUCED) {
    p = c.take(sizeof(double) * (size_t)n * n); if (D) D->gmat = (double*)p;
  }
  p = c.take(sizeof(double) * n);             if (D) D->gsc = (double*)p;
  p = c.take(sizeof(int) * 12);               if (D) D->arms_dev = (int*)p;
  p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->f = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->tmp = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->tmp2 = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->pbuf = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->rbuf = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->psave = (double*)p;
  p = c.take(sizeof(double) * nrhs);          if (D) D->fnorm0 = (double*)p;
  if (d->schur_mode == FPG_SCHUR_LITERAL) {
    p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->lit_in = (double*)p;
    p = c.take(sizeof(double) * nrhs * L.ntot); if (D) D->lit_out = (double*)p;
  } else if (D) {
    D->lit_in = D->lit_out = nullptr;
  }
  p = c.take(sizeof(double) * nrhs * std::max(4, L.narms) * n); if (D) D->corr = (double*)p;
  long long sc = (long long)nrhs * std::max(L.nc, 2 * L.na);
  if (L.lattice) {
    // the arm batches hold up to 8 blocks each; the coupled squares go 8 at a time
    const LatticeGeom& g = L.lg;
    sc = std::max(sc, (long long)nrhs * L.na * std::max(g.nwe, g.nsn));
    const long long nc = g.nc, nt = g.ntot;
    p = c.take(sizeof(int4) * nc);             if (D) D->lat.nbr = (const int4*)p;
    p = c.take(sizeof(int2) * nc);             if (D) D->lat.cf = (const int2*)p;
    p = c.take(sizeof(int2) * nc);             if (D) D->lat.anb = (const int2*)p;
    p = c.take(sizeof(int2) * std::max(1, g.nfaces)); if (D) D->lat.faces = (const int2*)p;
    p = c.take(sizeof(int4) * nt);             if (D) D->lat.gnbr = (const int4*)p;
    p = c.take(sizeof(int) * nt);              if (D) D->lat.gcn = (const int*)p;
    p = c.take(sizeof(double) * n);            if (D) D->lat.lpiv = (const double*)p;
    if (D) {
      D->lat.nc = nc;
      D->lat.link_base = g.link_base;
      D->lat.junc_base = g.junc_base;
      D->lat.nfaces = g.nfaces;
      D->lat.nlinks = g.nlinks;
      D->lat.njunc = g.njunc;
    }
  }
  p = c.take(sizeof(double) * sc);            if (D) D->scratch = p;
  p = c.take(sizeof(double) * nrhs);          if (D) D->gres = (double*)p;
  p = c.take(sizeof(int) * 4);                if (D) D->resume_dev = (int*)p;
  p = c.take(sizeof(int) * 4);                if (D) D->err_dev = (int*)p;
  KrylovState* k = D ? &D->ks : nullptr;
  p = c.take(sizeof(double) * (size_t)(m + 1) * nrhs * L.nc); if (k) k->V = (double*)p;
  p = c.take(zel * (size_t)m * nrhs * L.nc);                  if (k) k->Z = p;
  p = c.take(sizeof(double) * nrhs * L.nc);   if (k) k->w = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.nc);   if (k) k->u = (double*)p;
  p = c.take(sizeof(double) * nrhs * L.nc);   if (k) k->fc = (double*)p;
  p = c.take(sizeof(double) * (size_t)nrhs * m * (m + 1)); if (k) k->H = (double*)p;
  p = c.take(sizeof(double) * nrhs * m);      if (k) k->cs = (double*)p;
  p = c.take(sizeof(double) * nrhs * m);      if (k) k->sn = (double*)p;
  p = c.take(sizeof(double) * nrhs * (m + 1)); if (k) k->g = (double*)p;
  p = c.take(sizeof(double) * nrhs * m);      if (k) k->y = (double*)p;
  p = c.take(sizeof(double) * 2 * nrhs * kGmax); if (k) k->part = (double*)p;
  p = c.take(sizeof(double) * nrhs);          if (k) k->tolabs = (double*)p;
  p = c.take(sizeof(double) * nrhs);          if (k) k->fnorm = (double*)p;
  p = c.take(sizeof(double) * nrhs);          if (k) k->res = (double*)p;
  p = c.take(sizeof(double) * nrhs);          if (k) k->rnorm = (double*)p;
  p = c.take(sizeof(int) * nrhs);             if (k) k->active = (int*)p;
  p = c.take(sizeof(int) * nrhs);             if (k) k->done = (int*)p;
  p = c.take(sizeof(int) * nrhs);             if (k) k->kcyc = (int*)p;
  p = c.take(sizeof(int) * nrhs);             if (k) k->iters = (int*)p;
  // the one-pass FP32 cluster fast solve of the centre: sigma_k and the pivot at each strip start
  p = c.take(sizeof(float) * 17 * (size_t)n);
  if (D) {
    D->tC32.cl_sigma = p;
    D->tC32.cl_wseed = (const float*)p + n;
  }
}

// Phase timing helpers (only when profiling is on).  Events come from the
// direct-launch pool, or, while a restart cycle is being captured into a CUDA
// graph, from the graph's own pool (recorded again by every replay and read at
// the poll that follows it).
std::vector<cudaEvent_t>& ev_pool(fpg_domain* D) { return D->capturing ? D->gev : D->evpool; }
std::vector<std::pair<int, int>>& ev_list(fpg_domain* D) { return D->capturing ? D->gev_used : D->ev_used; }
int& ev_cursor(fpg_domain* D) { return D->capturing ? D->gev_next : D->ev_next; }

int ev_take(fpg_domain* D, int count) {
  if (!D->profiling || ev_cursor(D) + count > (int)ev_pool(D).size()) return -1;
  const int i = ev_cursor(D);
  ev_cursor(D) += count;
  return i;
}
// Inside a stream capture, cudaEventRecordExternal makes the record a graph node
// that records again at every replay (the flag is only legal while capturing).
void ev_record(fpg_domain* D, cudaEvent_t e) {
  if (D->capturing)
    cudaEventRecordWithFlags(e, D->st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, D->st);
}
int ev_begin(fpg_domain* D, int phase) {
  const int i = ev_take(D, 2);
  if (i < 0) return -1;
  ev_record(D, ev_pool(D)[i]);
  ev_list(D).push_back({phase, i});
  return i;
}
void ev_end(fpg_domain* D, int i) {
  if (i >= 0) ev_record(D, ev_pool(D)[i + 1]);
}
// Add the event pairs of the last graph replay to the phase totals.
void ev_collect_replay(fpg_domain* D) {
  if (!D->replay_pending) return;
  D->replay_pending = false;
  for (auto& pr : D->gev_used) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, D->gev[pr.second], D->gev[pr.second + 1]) == cudaSuccess)
      D->phase_ms[pr.first] += ms;
  }
  for (int i = 0; i < kPhases; ++i) D->phase_launches[i] += D->cycle_phase_launches[i];
}
void ev_collect(fpg_domain* D) {
  if (!D->profiling) return;
  cudaStreamSynchronize(D->st);
  ev_collect_replay(D);
  for (auto& pr : D->ev_used) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, D->evpool[pr.second], D->evpool[pr.second + 1]) == cudaSuccess)
      D->phase_ms[pr.first] += ms;
  }
  D->ev_used.clear();
  D->ev_next = 0;
}

inline void count(fpg_domain* D, int phase, int n) {
  D->launches += n;
  D->phase_launches[phase] += n;
}

// ---- building blocks used by the driver and the entry points ---------------

// a1 on nvec centre vectors (nvec <= nrhs): v (FP64, stride nc) -> z (prec).
fpg_status precond(fpg_domain* D, const double* v, void* z, int nvec, const int* active) {
  const Layout& L = D->L;
  if (L.chain && D->precond_kind == 0) {  // a chain's A_c: the coupled row's own operator, one fast solve
    int nl3 = 0;
    const BatchDesc rb{L.nc, {0, 0, 0, 0}, 1};
    FPG_CUDA_TRY(launch_fast_solve(D->prec, D->prec, D->prec == 64 ? D->tR64 : D->tR32, D->LR, v, rb, z, rb, nvec,
                                   D->scratch, active, 1, D->st, &nl3));
    count(D, 0, nl3);
    return FPG_OK;
  }
  if (D->precond_kind == 1 || D->precond_kind == 2) {  // Sec. 3.2 comparison preconditioners: identity, Jacobi
    FPG_CUDA_TRY(launch_precond_simple(v, z, D->prec, L.nc, L.n, D->delta, D->desc.kappa, D->ctab, L.armmask,
                                       D->precond_kind == 2, active, nvec, D->gx, D->st));
    count(D, 0, 1);
    return FPG_OK;
  }
  int nl = 0;
  if (L.lattice) {
    // block diagonal of the coupled set: the coupled squares' fast solves, 8 per
    // launch, then the links' and junctions' own operators
    const FastSolveTables& tc = D->prec == 64 ? D->tC64 : D->tC32;
    const LatticeGeom& g = L.lg;
    for (int k0 = 0; k0 < g.ncsq; k0 += 8) {
      BatchDesc bd{L.nc, {0, 0, 0, 0}, 0};
      for (int k = k0; k < g.ncsq && k < k0 + 8; ++k) bd.off[bd.nper++] = g.sq_off[k];
      FPG_CUDA_TRY(launch_fast_solve(D->prec, D->prec, tc, D->LC, v, bd, z, bd, nvec * bd.nper, D->scratch, active,
                                     bd.nper, D->st, &nl));
    }
    FPG_CUDA_TRY(launch_lattice_skeleton(v, z, D->prec, D->lat, L.n, D->delta, D->desc.kappa, active, nvec, D->st));
    count(D, 0, nl + 1);
    return FPG_OK;
  }
  if (L.chain) {  // FPG_OPT_PRECOND = 3
    // block-diagonal over the row's squares: 2K - 2 squares of n + 1 columns, then the last
    const FastSolveTables& ta = D->prec == 64 ? D->tA64 : D->tA32;
    const FastSolveTables& tc = D->prec == 64 ? D->tC64 : D->tC32;
    FPG_CUDA_TRY(launch_fast_solve(D->prec, D->prec, ta, D->LC1, v, D->cb1, z, D->cb1, nvec * D->cb1.nper,
                                   D->scratch, active, D->cb1.nper, D->st, &nl));
    FPG_CUDA_TRY(launch_fast_solve(D->prec, D->prec, tc, D->LC2, v, D->cb2, z, D->cb2, nvec, D->scratch, active, 1,
                                   D->st, &nl));
    count(D, 0, nl);
    return FPG_OK;
  }
  BatchDesc ib{L.nc, {0, 0, 0, 0}, 1};
  const FastSolveTables& tb = D->prec == 64 ? D->tC64 : D->tC32;
  cudaEvent_t* evp = nullptr;
  const int i = ev_take(D, 8);
  if (i >= 0) {
    // pool events i..i+7: start/end of the forward DST, the Thomas solve, the
    // inverse DST and the fused kernel (the path not taken records empty pairs)
    evp = &ev_pool(D)[i];
    ev_list(D).push_back({7, i});
    ev_list(D).push_back({8, i + 2});
    ev_list(D).push_back({9, i + 4});
    ev_list(D).push_back({10, i + 6});
  }
  FPG_CUDA_TRY(launch_fast_solve(D->prec, D->prec, tb, D->LC, v, ib, z, ib, nvec, D->scratch, active, 1, D->st,
                                 &nl, evp));
  count(D, 0, nl);
  if (evp) {
    if (nl == 1) {
      D->phase_launches[10] += 1;
    } else {
      D->phase_launches[7] += 1;
      D->phase_launches[8] += 1;
      D->phase_launches[9] += 1;
    }
  }
  return FPG_OK;
}

// FP64 fast solves on the arm blocks of nvec full vectors (in -> out), with the
// per-RHS flags `active` (may be null).  Vertex-centred arms: W and E in one
// batch, S and N in another (their sweeps are symmetric).  Neumann-sided arms:
// one batch per arm, since the far-end row is first in W and S and last in E
// and N, and the pivot tables differ.
cudaError_t arm_fast_solves(fpg_domain* D, const double* in, double* out, int nvec, const int* active, int* nl) {
  if (D->L.ao.bc == 0) {
    if (D->we.nper > 0) {
      const cudaError_t e = launch_fast_solve(64, 64, D->tA64, D->LWE, in, D->we, out, D->we, nvec * D->we.nper,
                                              D->scratch, active, D->we.nper, D->st, nl);
      if (e != cudaSuccess) return e;
    }
    for (const BatchDesc* g : {&D->sn, &D->sn2}) {  // sn2: a chain's N arms
      if (g->nper == 0) continue;
      const cudaError_t e = launch_fast_solve(64, 64, D->tA64, D->LSN, in, *g, out, *g, nvec * g->nper, D->scratch,
                                              active, g->nper, D->st, nl);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int a = 0; a < 4; ++a) {
    if (D->L.ao.off[a] < 0) continue;
    const BatchDesc bd{D->L.ntot, {D->L.ao.off[a], 0, 0, 0}, 1};
    const FastSolveTables& tb = (a == 0 || a == 2) ? D->tA64 : D->tA64e;
    const cudaError_t e = launch_fast_solve(64, 64, tb, a < 2 ? D->LWE : D->LSN, in, bd, out, bd, nvec, D->scratch,
                                            active, 1, D->st, nl);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Fast solves on the arms of nvec full vectors (FP64): in -> out (arm blocks only).
fpg_status arm_solves(fpg_domain* D, const double* in, double* out, int nvec, int phase) {
  int nl = 0;
  FPG_CUDA_TRY(arm_fast_solves(D, in, out, nvec, nullptr, &nl));
  count(D, phase, nl);
  return FPG_OK;
}

// Arm solves with one step of FP64 iterative refinement: out = A_a^{-1} in, then
// e = A_a^{-1}(in - A_a out), out += e.  The fast solve's forward error (DST
// rounding, ~1e-15..1e-14 relative) would otherwise leave a residual of about
// cond(A_a) times that in the global system; the refinement brings it down to
// the rounding of the residual evaluation itself.  `work` must not alias in/out.
fpg_status arm_solves_refined(fpg_domain* D, const double* in, double* out, double* work, int nvec, int phase) {
  const Layout& L = D->L;
  FPG_TRY(arm_solves(D, in, out, nvec, phase));
  // the arm kernels take up to four arms (W, E, S, N slots) per launch: the arms
  // of a chain or a lattice go group by group
  const int groups = (int)L.arm_groups.size();
  for (int it = 0; it < D->arm_refine && groups > 0; ++it) {  // out += A_a^{-1} (in - A_a out)
    for (const ArmOffsets& ao : L.arm_groups)
      FPG_CUDA_TRY(launch_arm_residual(in, out, work, L.ntot, L.n, D->delta, D->desc.kappa, ao, nvec, D->gxf, D->st));
    FPG_TRY(arm_solves(D, work, work, nvec, phase));
    for (const ArmOffsets& ao : L.arm_groups)
      FPG_CUDA_TRY(launch_arm_add(out, work, L.ntot, L.n, ao, nvec, D->gxf, D->st));
    count(D, phase, 2 * groups);
  }
  return FPG_OK;
}

// a2, interface part: corr[r][a][:] = R_ca A_a^{-1} R_ac z on C's line next to arm a.
fpg_status schur_corr(fpg_domain* D, const void* z, int zprec, int nvec, const int* active) {
  const Layout& L = D->L;
  if (L.chain) {
    FPG_CUDA_TRY(launch_chain_schur(z, zprec, L.nc, L.cg, D->ctab, D->corr, active, nvec, D->st));
    count(D, 1, 1);
    return FPG_OK;
  }
  if (D->desc.schur_mode == FPG_SCHUR_REDUCED) {
    if (D->schur_transform == 1 && L.ao.bc == 0 && schur_dst_supported(L.n))
      FPG_CUDA_TRY(launch_schur_dst(z, zprec, L.nc, L.n, D->tC64.plan, D->gsc, D->arms_dev, L.narms, D->corr, active,
                                    nvec, D->st));
    else if (D->schur_transform == 0 && D->gmat != nullptr)
      FPG_CUDA_TRY(launch_schur_gmat(z, zprec, L.nc, L.n, D->gmat, D->arms_dev, L.narms, D->corr, active, nvec,
                                     D->st));
    else
      FPG_CUDA_TRY(launch_schur_reduced(z, zprec, L.nc, L.n, D->ctab, D->arms_dev, L.narms, D->corr, active, nvec,
                                        D->st));
    count(D, 1, 1);
  } else {
    FPG_CUDA_TRY(launch_literal_inject(z, zprec, L.nc, L.n, D->delta, D->lit_in, L.ntot, L.ao, active, nvec,
                                       D->gxf, D->st));
    count(D, 1, 1);
    int nl = 0;
    FPG_CUDA_TRY(arm_fast_solves(D, D->lit_in, D->lit_out, nvec, active, &nl));
    count(D, 1, nl);
    FPG_CUDA_TRY(launch_literal_extract(D->lit_out, L.ntot, L.ao, L.n, D->delta, D->corr, active, nvec, D->st));
    count(D, 1, 1);
  }
  return FPG_OK;
}

// a2 on nvec centre vectors (nvec <= nrhs): z (zprec) -> w.
fpg_status schur(fpg_domain* D, const void* z, int zprec, double* w, int nvec, const int* active) {
  const Layout& L = D->L;
  if (L.lattice) {
    FPG_CUDA_TRY(launch_lattice_schur(z, zprec, L.nc, w, L.nc, D->lat, L.n, D->delta, D->desc.kappa, D->ctab,
                                      D->corr, active, nvec, D->gx, D->st));
    count(D, 1, D->lat.nfaces > 0 ? 2 : 1);
    return FPG_OK;
  }
  FPG_TRY(schur_corr(D, z, zprec, nvec, active));
  if (L.chain)
    FPG_CUDA_TRY(launch_chain_stencil(z, zprec, L.nc, w, L.nc, L.cg, D->delta, D->desc.kappa, D->corr, active, nvec,
                                      D->gx, D->st));
  else
    FPG_CUDA_TRY(launch_stencil_c(z, zprec, L.nc, w, L.nc, L.n, D->delta, D->desc.kappa, D->corr, L.armmask,
                                  active, nvec, D->gx, D->st));
  count(D, 1, 1);
  return FPG_OK;
}

// a7: y = K p (y may be null) and, with f, the relative residuals ||f - K p||/||f||.
cudaError_t global_apply(fpg_domain* D, const double* p, double* y, const double* f, int nvec, double* rel_out,
                         double* fnorm_out, double rtol, double* tolabs) {
  const Layout& L = D->L;
  if (L.lattice)
    return launch_lattice_global_apply(p, y, f, L.ntot, D->lat, D->delta, D->desc.kappa, D->ks.part, kGmax, nvec,
                                       D->gxf, rel_out, fnorm_out, rtol, tolabs, D->st);
  if (L.chain)
    return launch_chain_global_apply(p, y, f, L.ntot, L.cg, D->delta, D->desc.kappa, D->ks.part, kGmax, nvec, D->gxf,
                                     rel_out, fnorm_out, rtol, tolabs, D->st);
  return launch_global_apply(p, y, f, L.ntot, L.n, D->delta, D->desc.kappa, L.ao, D->ks.part, kGmax, nvec, D->gxf,
                             rel_out, fnorm_out, rtol, tolabs, D->st);
}

fpg_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    record_cuda_error(e, "kernel launch");
    return FPG_ECUDA;
  }
  return FPG_OK;
}


// The solve in stages, so that several domains can be interleaved from one host
// thread: setup (Alg. 1 steps 1-3), restart (true residual, restart flags and an
// asynchronous read of the "done" flags into pinned host memory), poll (wait
// for that read), cycle (m Arnoldi steps and the cycle end), finish (Alg. 1
// steps 5-7 and the acceptance residual).  The only host synchronisation is
// the poll, once per restart cycle.
// Setup on D->f into p (Alg. 1 steps 1-3); keep_iters: a refinement solve
// continues the iteration counts of the solve it corrects.
fpg_status setup_common(fpg_domain* D, double* p, bool keep_iters);

fpg_status stage_setup(fpg_domain* D, double* p) {
  FPG_CUDA_TRY(cudaMemsetAsync(D->err_dev, 0, sizeof(int), D->st));
  D->cycles_run = 0;
  D->accept_rounds = 0;
  D->refining = false;
  D->p_cur = p;
  FPG_TRY(setup_common(D, p, false));
  // ||f|| of the caller's right-hand sides, the scale of every later acceptance test
  FPG_CUDA_TRY(cudaMemcpyAsync(D->fnorm0, D->ks.fnorm, sizeof(double) * D->desc.nrhs, cudaMemcpyDeviceToDevice,
                               D->st));
  return FPG_OK;
}

fpg_status setup_common(fpg_domain* D, double* p, bool keep_iters) {
  const Layout& L = D->L;
  KrylovState& k = D->ks;
  const int nrhs = D->desc.nrhs;
  D->first_cycle = true;
  // ||f|| per RHS and the absolute tolerance
  int e = ev_begin(D, 5);
  FPG_CUDA_TRY(global_apply(D, D->f, nullptr, D->f, nrhs, nullptr, k.fnorm, kInnerMargin * D->desc.rtol, k.tolabs));
  count(D, 5, 2);
  // Alg. 1 steps 1-3: q_a = A_a^{-1} f_a (into p's arm blocks), f'_c = f_c - sum R_ca q_a
  FPG_TRY(arm_solves_refined(D, D->f, p, D->tmp2, nrhs, 5));
  if (L.lattice)
    FPG_CUDA_TRY(launch_lattice_reduce_rhs(D->f, p, L.ntot, D->lat, D->delta, k.fc, nrhs, D->gx, D->st));
  else if (L.chain)
    FPG_CUDA_TRY(launch_chain_reduce_rhs(D->f, p, L.ntot, L.cg, D->delta, k.fc, nrhs, D->gx, D->st));
  else
    FPG_CUDA_TRY(launch_reduce_rhs(D->f, p, L.ntot, L.n, D->delta, L.ao, k.fc, nrhs, D->gx, D->st));
  count(D, 5, 1);
  FPG_CUDA_TRY(cudaMemsetAsync(k.u, 0, sizeof(double) * nrhs * L.nc, D->st));
  FPG_CUDA_TRY(cudaMemsetAsync(k.done, 0, sizeof(int) * nrhs, D->st));
  if (!keep_iters) FPG_CUDA_TRY(cudaMemsetAsync(k.iters, 0, sizeof(int) * nrhs, D->st));
  FPG_CUDA_TRY(cudaMemsetAsync(k.w, 0, sizeof(double) * nrhs * L.nc, D->st));
  ev_end(D, e);
  return FPG_OK;
}

fpg_status stage_restart(fpg_domain* D) {
  const Layout& L = D->L;
  KrylovState& k = D->ks;
  const int nrhs = D->desc.nrhs, m = D->desc.restart;
  // restart: w = L_c u (skipped while u = 0), r = f'_c - w -> V[0], beta, flags
  int e = ev_begin(D, 4);
  if (!D->first_cycle) FPG_TRY(schur(D, k.u, 64, k.w, nrhs, nullptr));
  FPG_CUDA_TRY(launch_restart(k.fc, k.w, k.V, L.nc, nrhs, k.part, kGmax, k.g, m, k.tolabs, k.rnorm, k.done, k.active,
                              k.kcyc, k.iters, D->desc.max_iters, D->gx, D->st));
  count(D, 4, 2);
  ev_end(D, e);
  D->first_cycle = false;
  FPG_CUDA_TRY(cudaMemcpyAsync(D->h_done_pinned, k.done, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, D->st));
  FPG_CUDA_TRY(cudaEventRecord(D->ev_flags, D->st));
  return FPG_OK;
}

fpg_status stage_poll(fpg_domain* D, bool* all_done) {
  FPG_CUDA_TRY(cudaEventSynchronize(D->ev_flags));
  ev_collect_replay(D);
  bool all = true;
  for (int r = 0; r < D->desc.nrhs; ++r) all = all && D->h_done_pinned[r];
  const int max_cycles = (D->desc.max_iters + D->desc.restart - 1) / D->desc.restart + 2;
  *all_done = all || D->cycles_run >= max_cycles;
  return FPG_OK;
}

fpg_status issue_cycle(fpg_domain* D) {
  const Layout& L = D->L;
  KrylovState& k = D->ks;
  const int nrhs = D->desc.nrhs, m = D->desc.restart;
  const int hcol = m + 1, hrhs = m * (m + 1);
  const int zprec = D->prec;
  const size_t zel = zprec == 64 ? 8 : 4;
  int e;
  for (int j = 0; j < m; ++j) {
    double* vj = k.V + (size_t)j * nrhs * L.nc;
    void* zj = (char*)k.Z + zel * (size_t)j * nrhs * L.nc;
    e = ev_begin(D, 0);
    FPG_TRY(precond(D, vj, zj, nrhs, k.active));
    ev_end(D, e);
    const int csz = D->use_cluster ? (D->tune_csz > 0 ? D->tune_csz : arnoldi_cluster_size(L.nc)) : 0;
    // the register-resident step fuses the cross's stencil: chains take the global-w step
    const int ept = (csz > 0 && D->arnoldi_mode == 1 && !L.chain && !L.lattice)
                        ? arnoldi_reg_ept(L.nc, csz, D->tune_nt) : 0;
    if (ept > 0) {
      // a2's interface part, then one launch for a2's stencil + a3 + a4
      e = ev_begin(D, 1);
      FPG_TRY(schur_corr(D, zj, zprec, nrhs, k.active));
      ev_end(D, e);
      e = ev_begin(D, 2);
      FPG_CUDA_TRY(launch_arnoldi_reg(csz, D->tune_nt, k.V, (long long)nrhs * L.nc, nullptr, zj, zprec, D->corr, L.n, D->delta,
                                      D->desc.kappa, L.armmask, k.V + (size_t)(j + 1) * nrhs * L.nc, L.nc, j, nrhs,
                                      k.H, hcol, hrhs, k.cs, k.sn, k.g, k.res, m, k.tolabs, k.active, k.kcyc,
                                      k.iters, D->desc.max_iters, 1, D->err_dev, D->st));
      count(D, 2, 1);
      ev_end(D, e);
      if (D->hist) {
        FPG_CUDA_TRY(launch_record_history(k.res, k.iters, D->hist, D->hist_len, nrhs, D->st));
        count(D, 3, 1);
      }
      continue;
    }
    e = ev_begin(D, 1);
    FPG_TRY(schur(D, zj, zprec, k.w, nrhs, k.active));
    ev_end(D, e);
    e = ev_begin(D, 2);
    if (csz > 0) {
      // a3 + a4 fused: one cluster per right-hand side
      FPG_CUDA_TRY(launch_arnoldi_cluster(csz, k.V, (long long)nrhs * L.nc, k.w, k.V + (size_t)(j + 1) * nrhs * L.nc,
                                          L.nc, j, nrhs, k.H, hcol, hrhs, k.cs, k.sn, k.g, k.res, m, k.tolabs,
                                          k.active, k.kcyc, k.iters, D->desc.max_iters, 1, D->st));
      count(D, 2, 1);
      ev_end(D, e);
    } else {
      int nl = 0;
      FPG_CUDA_TRY(launch_mgs(k.V, (long long)nrhs * L.nc, k.w, k.V + (size_t)(j + 1) * nrhs * L.nc, L.nc, j, nrhs,
                              k.part, kGmax, k.H, hcol, hrhs, k.active, D->gx, D->st, &nl));
      count(D, 2, nl);
      ev_end(D, e);
      e = ev_begin(D, 3);
      FPG_CUDA_TRY(launch_givens(k.H, hcol, hrhs, k.cs, k.sn, k.g, k.res, j, m, nrhs, k.tolabs, k.active, k.kcyc,
                                 k.iters, D->desc.max_iters, D->st));
      count(D, 3, 1);
      ev_end(D, e);
    }
    if (D->hist) {
      FPG_CUDA_TRY(launch_record_history(k.res, k.iters, D->hist, D->hist_len, nrhs, D->st));
      count(D, 3, 1);
    }
  }
  e = ev_begin(D, 4);
  FPG_CUDA_TRY(launch_cycle_end(k.H, hcol, hrhs, k.g, k.y, m, nrhs, k.kcyc, k.u, k.Z, zprec, (long long)nrhs * L.nc,
                                L.nc, D->gx, D->st));
  count(D, 4, 2);
  ev_end(D, e);
  return FPG_OK;
}

// Drop the captured cycle (after anything that changes the launch sequence).
void drop_graph(fpg_domain* D) {
  if (D->cycle_exec) cudaGraphExecDestroy(D->cycle_exec);
  D->cycle_exec = nullptr;
}

// One restart cycle.  Every cycle of a domain issues the same launches with the
// same arguments (right-hand sides that converge switch off through the device
// "active" flags), so the cycle is captured once into a CUDA graph and replayed:
// one launch per cycle instead of ~5 per Arnoldi step.  Not used while
// profiling (the per-phase events are host-recorded) or on the legacy default
// stream, which cannot be captured.
fpg_status stage_cycle(fpg_domain* D) {
  D->cycles_run++;
  if (!D->use_graphs || D->st == nullptr) return issue_cycle(D);
  if (D->cycle_exec && D->graph_profiled != D->profiling) drop_graph(D);
  if (!D->cycle_exec) {
    const long long before = D->launches;
    long long ph_before[kPhases];
    for (int i = 0; i < kPhases; ++i) ph_before[i] = D->phase_launches[i];
    if (D->profiling && D->gev.empty()) {
      D->gev.resize(12 * D->desc.restart + 8);
      for (auto& ev : D->gev) FPG_CUDA_TRY(cudaEventCreate(&ev));
    }
    D->gev_used.clear();
    D->gev_next = 0;
    D->capturing = true;
    cudaGraph_t graph = nullptr;
    cudaError_t be = cudaStreamBeginCapture(D->st, cudaStreamCaptureModeThreadLocal);
    if (be != cudaSuccess) {
      D->capturing = false;
      record_cuda_error(be, "cudaStreamBeginCapture");
      return FPG_ECUDA;
    }
    const fpg_status st = issue_cycle(D);
    const cudaError_t ce = cudaStreamEndCapture(D->st, &graph);
    D->capturing = false;
    for (int i = 0; i < kPhases; ++i) {
      D->cycle_phase_launches[i] = D->phase_launches[i] - ph_before[i];
      D->phase_launches[i] = ph_before[i];
    }
    D->graph_profiled = D->profiling;
    if (st != FPG_OK || ce != cudaSuccess) {
      // Nothing of a failed capture ran.  A capture can be invalidated from
      // outside (work another thread put on the same stream, a device-wide
      // synchronisation): clear the error, give up graphs on this domain and
      // issue the cycle directly.
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      D->launches = before;
      D->use_graphs = false;
      if (st != FPG_OK && st != FPG_ECUDA) return st;
      return issue_cycle(D);
    }
    const cudaError_t ie = cudaGraphInstantiate(&D->cycle_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      D->cycle_exec = nullptr;
      record_cuda_error(ie, "cudaGraphInstantiate");
      return FPG_ECUDA;
    }
    D->cycle_kernels = D->launches - before;  // kernels in one replay
    D->launches = before;
  }
  FPG_CUDA_TRY(cudaGraphLaunch(D->cycle_exec, D->st));
  D->launches += D->cycle_kernels;
  if (D->graph_profiled) D->replay_pending = true;
  return FPG_OK;
}

fpg_status stage_finish(fpg_domain* D) {
  const Layout& L = D->L;
  KrylovState& k = D->ks;
  const int nrhs = D->desc.nrhs;
  double* p = D->p_cur;
  // Alg. 1 steps 5-7: f'_a = f_a - R_ac p_c, p_a = A_a^{-1} f'_a, p_c = u
  int e = ev_begin(D, 5);
  if (L.lattice)
    FPG_CUDA_TRY(launch_lattice_arm_rhs(D->f, k.u, L.ntot, D->lat, D->delta, D->tmp, p, nrhs, D->gxf, D->st));
  else if (L.chain)
    FPG_CUDA_TRY(launch_chain_arm_rhs(D->f, k.u, L.ntot, L.cg, D->delta, D->tmp, p, nrhs, D->gxf, D->st));
  else
    FPG_CUDA_TRY(launch_arm_rhs(D->f, k.u, L.ntot, L.n, D->delta, L.ao, D->tmp, p, nrhs, D->gxf, D->st));
  count(D, 5, 1);
  FPG_TRY(arm_solves_refined(D, D->tmp, p, D->tmp2, nrhs, 5));
  ev_end(D, e);
  // a7: global relative residual, always against the caller's f
  e = ev_begin(D, 6);
  if (D->refining) {  // p held the correction: p = saved iterate + correction
    FPG_CUDA_TRY(launch_add_vec(p, D->psave, (long long)nrhs * L.ntot, D->st));
    D->f = D->f_orig;
    D->refining = false;
    count(D, 6, 1);
  }
  const bool check = D->accept_rounds < kAcceptRounds;
  // with a check to follow, K p goes to rbuf (the next refinement's residual)
  FPG_CUDA_TRY(global_apply(D, p, check ? D->rbuf : nullptr, D->f, nrhs, D->gres, nullptr, 0.0, nullptr));
  count(D, 6, 2);
  // acceptance check: right-hand sides still above rtol get r = f - K p for a
  // correction solve (global iterative refinement); the others get r = 0
  D->accept_rounds++;
  if (check) {
    FPG_CUDA_TRY(cudaMemsetAsync(D->resume_dev, 0, sizeof(int), D->st));
    FPG_CUDA_TRY(launch_refine_rhs(D->f, D->rbuf, D->gres, D->desc.rtol, L.ntot, nrhs, D->resume_dev, D->gxf, D->st));
    count(D, 6, 1);
    FPG_CUDA_TRY(cudaMemcpyAsync(D->h_done_pinned + nrhs, D->resume_dev, sizeof(int), cudaMemcpyDeviceToHost, D->st));
  }
  ev_end(D, e);
  FPG_CUDA_TRY(cudaEventRecord(D->ev_flags, D->st));
  return check_launch();
}

// After stage_finish: does any right-hand side resume (waits for the check)?
// A resume is one step of global iterative refinement: the same Alg. 1 run on
// r = f - K p (setup, FGMRES cycles, finish) gives a correction that the next
// stage_finish adds to the saved iterate.  Its Krylov target is absolute,
// 0.45 rtol ||f|| with the caller's f, so the correction needs only a few
// iterations; it also corrects the setup's f'_c, whose rounding sets a floor
// that a tighter Schur target alone does not move (seen at n = 1024).
fpg_status stage_resume(fpg_domain* D, bool* resume) {
  *resume = false;
  if (D->accept_rounds > kAcceptRounds) return FPG_OK;
  FPG_CUDA_TRY(cudaEventSynchronize(D->ev_flags));
  *resume = D->h_done_pinned[D->desc.nrhs] > 0;
  if (!*resume) return FPG_OK;
  const int nrhs = D->desc.nrhs;
  double* p = D->p_cur;
  FPG_CUDA_TRY(cudaMemcpyAsync(D->psave, p, sizeof(double) * nrhs * D->L.ntot, cudaMemcpyDeviceToDevice, D->st));
  D->f_orig = D->f;
  D->f = D->rbuf;
  D->refining = true;
  FPG_TRY(setup_common(D, p, true));
  FPG_CUDA_TRY(launch_refine_tol(D->ks.tolabs, D->fnorm0, 0.5 * kInnerMargin * D->desc.rtol, nrhs, D->st));
  count(D, 5, 1);
  return FPG_OK;
}

// One domain, start to finish (the host waits once per restart cycle, and once
// per acceptance check).
// Setup of a solve that starts from the iterate held in p (checkpoint / resume):
// r = f - K p for the right-hand sides whose relative residual is above rtol
// (0 for the others), then the same algorithm on r, whose result is added to
// the saved iterate at finish -- the machinery of the acceptance loop's global
// refinement, with the Krylov target 0.9 rtol ||f||.
fpg_status stage_setup_from(fpg_domain* D, double* p) {
  const Layout& L = D->L;
  const int nrhs = D->desc.nrhs;
  FPG_CUDA_TRY(cudaMemsetAsync(D->err_dev, 0, sizeof(int), D->st));
  D->cycles_run = 0;
  D->accept_rounds = 0;
  D->refining = false;
  D->p_cur = p;
  int e = ev_begin(D, 6);
  FPG_CUDA_TRY(global_apply(D, p, D->rbuf, D->f, nrhs, D->gres, D->fnorm0, 0.0, nullptr));
  FPG_CUDA_TRY(cudaMemsetAsync(D->resume_dev, 0, sizeof(int), D->st));
  FPG_CUDA_TRY(launch_refine_rhs(D->f, D->rbuf, D->gres, D->desc.rtol, L.ntot, nrhs, D->resume_dev, D->gxf, D->st));
  FPG_CUDA_TRY(cudaMemcpyAsync(D->psave, p, sizeof(double) * nrhs * L.ntot, cudaMemcpyDeviceToDevice, D->st));
  count(D, 6, 3);
  ev_end(D, e);
  D->f_orig = D->f;
  D->f = D->rbuf;
  D->refining = true;
  FPG_TRY(setup_common(D, p, false));
  FPG_CUDA_TRY(launch_refine_tol(D->ks.tolabs, D->fnorm0, kInnerMargin * D->desc.rtol, nrhs, D->st));
  count(D, 5, 1);
  return FPG_OK;
}

fpg_status solve_launch(fpg_domain* D, double* p, bool from_p = false) {
  FPG_TRY(from_p ? stage_setup_from(D, p) : stage_setup(D, p));
  for (;;) {
    for (;;) {
      FPG_TRY(stage_restart(D));
      bool done = false;
      FPG_TRY(stage_poll(D, &done));
      if (done) break;
      FPG_TRY(stage_cycle(D));
    }
    FPG_TRY(stage_finish(D));
    bool resume = false;
    FPG_TRY(stage_resume(D, &resume));
    if (!resume) return FPG_OK;
  }
}

fpg_status collect_info(fpg_domain* D, fpg_solve_info* info) {
  const int nrhs = D->desc.nrhs;
  std::vector<double> gres(nrhs), res(nrhs), fn(nrhs), rn(nrhs);
  std::vector<int> iters(nrhs), done(nrhs);
  KrylovState& k = D->ks;
  FPG_CUDA_TRY(cudaMemcpyAsync(gres.data(), D->gres, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, D->st));
  FPG_CUDA_TRY(cudaMemcpyAsync(rn.data(), k.rnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, D->st));
  FPG_CUDA_TRY(cudaMemcpyAsync(fn.data(), k.fnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, D->st));
  FPG_CUDA_TRY(cudaMemcpyAsync(iters.data(), k.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, D->st));
  int waited_out = 0;
  FPG_CUDA_TRY(cudaMemcpyAsync(&waited_out, D->err_dev, sizeof(int), cudaMemcpyDeviceToHost, D->st));
  FPG_CUDA_TRY(cudaStreamSynchronize(D->st));
  ev_collect(D);
  fpg_status all = waited_out ? FPG_ETIMEOUT : FPG_OK;
  for (int r = 0; r < nrhs; ++r) {
    const bool ok = gres[r] <= D->desc.rtol;
    // a device wait that gave up left part of a fast solve undone: every
    // right-hand side of the solve reports it, whatever its residual
    const fpg_status s = waited_out ? FPG_ETIMEOUT : ok ? FPG_OK : FPG_ENOCONV;
    if (s == FPG_ENOCONV && all == FPG_OK) all = FPG_ENOCONV;
    if (info) {
      info[r].iterations = iters[r];
      info[r].restarts = D->cycles_run;
      info[r].status = s;
      info[r].reserved = 0;
      info[r].residual = gres[r];
      info[r].schur_residual = fn[r] > 0 ? rn[r] / fn[r] : rn[r];
    }
  }
  return all;
}

}  // namespace

// ---- the staged solve without host waits (used by the batch runtime) --------
namespace fpg {

// Start a solve of the domain's right-hand sides into p (setup and the first
// restart are issued on the domain's stream).
fpg_status batch_start(fpg_domain* D, double* p) {
  FPG_TRY(stage_setup(D, p));
  FPG_TRY(stage_restart(D));
  D->bphase = 1;
  return FPG_OK;
}

// Has the work the host waits for next (restart flags or acceptance check) finished?
bool batch_ready(fpg_domain* D) { return cudaEventQuery(D->ev_flags) == cudaSuccess; }

// Advance a ready domain by one stage; *finished when its results are final.
fpg_status batch_advance(fpg_domain* D, bool* finished) {
  *finished = false;
  if (D->bphase == 1) {
    bool done = false;
    FPG_TRY(stage_poll(D, &done));
    if (done) {
      FPG_TRY(stage_finish(D));
      D->bphase = 2;
    } else {
      FPG_TRY(stage_cycle(D));
      FPG_TRY(stage_restart(D));
    }
  } else if (D->bphase == 2) {
    bool resume = false;
    FPG_TRY(stage_resume(D, &resume));
    if (resume) {
      FPG_TRY(stage_restart(D));
      D->bphase = 1;
    } else {
      D->bphase = 0;
      *finished = true;
    }
  }
  return FPG_OK;
}

fpg_status batch_info(fpg_domain* D, fpg_solve_info* info) { return collect_info(D, info); }

// Zero right-hand-side slots first..nrhs-1 (they converge before the first Arnoldi step).
fpg_status batch_zero_rhs(fpg_domain* D, int first) {
  if (first >= D->desc.nrhs) return FPG_OK;
  const size_t one = sizeof(double) * D->L.ntot;
  FPG_CUDA_TRY(cudaMemsetAsync(D->f + (size_t)first * D->L.ntot, 0, one * (D->desc.nrhs - first), D->st));
  return FPG_OK;
}

}  // namespace fpg

extern "C" {

const char* fpg_status_string(fpg_status s) {
  switch (s) {
    case FPG_OK: return "FPG_OK";
    case FPG_EINVAL: return "FPG_EINVAL: invalid argument";
    case FPG_ENOMEM: return "FPG_ENOMEM: workspace too small";
    case FPG_ECUDA: return "FPG_ECUDA: CUDA error";
    case FPG_ENOCONV: return "FPG_ENOCONV: not converged";
    case FPG_ETIMEOUT: return "FPG_ETIMEOUT: device wait gave up";
    case FPG_EUNSUPPORTED: return "FPG_EUNSUPPORTED";
    case FPG_EBUDGET: return "FPG_EBUDGET: over the memory budget";
  }
  return "unknown status";
}

const char* fpg_last_cuda_error(void) { return g_last_err; }
const char* fpg_version(void) { return "fpg 0.1 (sm_103a)"; }

fpg_status fpg_unknowns(const fpg_domain_desc* desc, int64_t* count) {
  if (!count) return FPG_EINVAL;
  FPG_TRY(validate(desc));
  Layout L;
  make_layout(desc, &L);
  *count = L.ntot;
  return FPG_OK;
}

fpg_status fpg_workspace_bytes(const fpg_domain_desc* desc, size_t* bytes) {
  if (!bytes) return FPG_EINVAL;
  FPG_TRY(validate(desc));
  Layout L;
  make_layout(desc, &L);
  HostPlan hp = plan_shape(desc->n);
  Carver c(nullptr);
  carve(nullptr, desc, L, &hp, c);
  *bytes = c.used + 256;
  return FPG_OK;
}

fpg_status fpg_create_domain(const fpg_domain_desc* desc, void* ws, size_t bytes, void* stream, fpg_domain** out) {
  if (!out || !ws) return FPG_EINVAL;
  *out = nullptr;
  FPG_TRY(validate(desc));
  size_t need = 0;
  fpg_workspace_bytes(desc, &need);
  if (bytes < need) return FPG_ENOMEM;
  fpg_domain* D = new (std::nothrow) fpg_domain();
  if (!D) return FPG_ENOMEM;
  D->desc = *desc;
  make_layout(desc, &D->L);
  const Layout& L = D->L;
  const int n = desc->n;
  D->st = (cudaStream_t)stream;
  const int as = L.ao.as;  // arm sweep length: n + 1 (vertex-centred) or n (cell-centred)
  const bool nside = L.ao.bc == 1;
  D->delta = nside ? (double)n * (double)n : (double)(n + 1) * (double)(n + 1);
  D->prec = desc->precond_precision;
  D->LC = LineLayout{n, n, 1, n};
  D->LWE = LineLayout{n, as, as, 1};
  D->LSN = LineLayout{n, as, 1, n};
  D->we = BatchDesc{L.ntot, {0, 0, 0, 0}, 0};
  D->sn = BatchDesc{L.ntot, {0, 0, 0, 0}, 0};
  D->sn2 = BatchDesc{L.ntot, {0, 0, 0, 0}, 0};
  if (L.chain) {
    const int K = L.chain, nxc = L.cg.nxc;
    D->we.off[D->we.nper++] = L.cg.off[0];
    D->we.off[D->we.nper++] = L.cg.off[1];
    for (int i = 0; i < K; ++i) {
      D->sn.off[D->sn.nper++] = L.cg.off[2 + i];
      D->sn2.off[D->sn2.nper++] = L.cg.off[2 + K + i];
    }
    // the row's squares: transform along y (stride nxc), sweep along x
    D->LC1 = LineLayout{n, n + 1, nxc, 1};
    D->LC2 = LineLayout{n, n, nxc, 1};
    D->cb1 = BatchDesc{L.nc, {0, 0, 0, 0}, 0};
    for (int q = 0; q < 2 * K - 2; ++q) D->cb1.off[D->cb1.nper++] = (long long)q * (n + 1);
    D->cb2 = BatchDesc{L.nc, {(long long)(2 * K - 2) * (n + 1), 0, 0, 0}, 1};
    D->LR = LineLayout{n, nxc, nxc, 1};
  } else if (L.lattice) {
    for (int k = 0; k < L.lg.nwe; ++k) D->we.off[D->we.nper++] = L.lg.we_off[k];
    for (int k = 0; k < L.lg.nsn; ++k) D->sn.off[D->sn.nper++] = L.lg.sn_off[k];
  } else {
    for (int a = 0; a < 4; ++a) {
      if (L.ao.off[a] < 0) continue;
      BatchDesc& g = a < 2 ? D->we : D->sn;
      g.off[g.nper++] = L.ao.off[a];
    }
  }
  for (auto* t : {&D->tC64, &D->tC32}) { t->n = n; t->ns = n; t->delta = D->delta; }
  for (auto* t : {&D->tA64, &D->tA32, &D->tA64e}) { t->n = n; t->ns = as; t->delta = D->delta; }
  for (auto* t : {&D->tR64, &D->tR32}) { t->n = n; t->ns = L.chain ? L.cg.nxc : 0; t->delta = D->delta; }
  HostPlan hp = build_plan(n);
  Carver c(ws);
  carve(D, desc, L, &hp, c);
  for (auto* t : {&D->tC64, &D->tC32, &D->tA64, &D->tA32, &D->tA64e, &D->tR64, &D->tR32}) t->err = D->err_dev;
  const int nrhs = desc->nrhs;
  D->gx = pick_gx(L.nc, nrhs);
  D->gxf = pick_gx(L.ntot, nrhs);
  D->ks.nrhs = nrhs;
  D->ks.m = desc->restart;
  D->ks.n = n;
  D->ks.nc = L.nc;
  D->ks.gx = D->gx;
  D->h_done.assign(nrhs, 0);
  // host tables
  std::vector<double> pc, pa, ct, ma, pae, mae, Wd, postd;
  std::vector<float> cl_sigma, cl_wseed;
  std::vector<double> gs(n, 0.0);
  fill_pivots(n, n, D->delta, desc->kappa, pc);
  if (!nside) {
    fill_pivots(n, n + 1, D->delta, desc->kappa, pa);
    fill_ctab(n, D->delta, pa, ct);
    for (int k = 1; k <= n; ++k) gs[k - 1] = pa[(size_t)(k - 1) * (n + 1) + n] * D->delta * D->delta / (2.0 * (n + 1));
    ma.resize(pa.size());
    for (size_t i = 0; i < pa.size(); ++i) ma[i] = -D->delta * pa[i];
  } else {
    // the far end is a Dirichlet face half a cell beyond row 0 (W, S) or row n-1 (E, N)
    dct_pivots(n, n, D->delta, desc->kappa, -D->delta, 0, pa, ma);
    dct_pivots(n, n, D->delta, desc->kappa, -D->delta, 1, pae, mae);
    dct_tables(n, Wd, postd);
    fill_ctab_dct(n, D->delta, pa, ct);
  }
  std::vector<float> pc32(pc.begin(), pc.end()), pa32(pa.begin(), pa.end());
  std::vector<double> mc(pc.size());
  for (size_t i = 0; i < pc.size(); ++i) mc[i] = -D->delta * pc[i];
  std::vector<float> mc32(mc.begin(), mc.end()), ma32(ma.begin(), ma.end());
  std::vector<float> W32(hp.W.begin(), hp.W.end()), s32(hp.sinp.begin(), hp.sinp.end()),
      B32(hp.Bhat.begin(), hp.Bhat.end()), d32(hp.dense.begin(), hp.dense.end());
  int arms[12] = {0};
  for (int i = 0; i < L.narms && i < 12; ++i) arms[i] = L.chain ? i : L.arm_slots[i % 4];
  auto cp = [&](const void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(const_cast<void*>(dst), src, b, cudaMemcpyHostToDevice, D->st);
  };
  cudaError_t err = cudaSuccess;
  {
    const DstPlan& p64 = D->tC64.plan;
    const DstPlan& p32 = D->tC32.plan;
    if (!err) err = cp(p64.W, hp.W.data(), sizeof(double) * hp.W.size());
    if (!err) err = cp(p32.W, W32.data(), sizeof(float) * W32.size());
    if (!err) err = cp(p64.sinp, hp.sinp.data(), sizeof(double) * hp.sinp.size());
    if (!err) err = cp(p32.sinp, s32.data(), sizeof(float) * s32.size());
    if (!err) err = cp(p64.dense, hp.dense.data(), sizeof(double) * hp.dense.size());
    if (!err) err = cp(p32.dense, d32.data(), sizeof(float) * d32.size());
    if (hp.mode == DST_RADER) {
      if (!err) err = cp(p64.Bhat, hp.Bhat.data(), sizeof(double) * hp.Bhat.size());
      if (!err) err = cp(p32.Bhat, B32.data(), sizeof(float) * B32.size());
      if (!err) err = cp(p64.pin, hp.pin.data(), sizeof(int) * hp.pin.size());
      if (!err) err = cp(p64.pout, hp.pout.data(), sizeof(int) * hp.pout.size());
      if (!err) err = cp(p32.pin, hp.pin.data(), sizeof(int) * hp.pin.size());
      if (!err) err = cp(p32.pout, hp.pout.data(), sizeof(int) * hp.pout.size());
    }
  }
  if (!err) err = cp(D->tC64.rpiv, pc.data(), sizeof(double) * pc.size());
  if (!err) err = cp(D->tC32.rpiv, pc32.data(), sizeof(float) * pc32.size());
  if (!err) err = cp(D->tA64.rpiv, pa.data(), sizeof(double) * pa.size());
  if (!err) err = cp(D->tA32.rpiv, pa32.data(), sizeof(float) * pa32.size());
  if (!err) err = cp(D->tC64.mneg, mc.data(), sizeof(double) * mc.size());
  if (!err) err = cp(D->tC32.mneg, mc32.data(), sizeof(float) * mc32.size());
  if (!err) err = cp(D->tA64.mneg, ma.data(), sizeof(double) * ma.size());
  {
    std::vector<double> pf, pb;
    thomas_chunk_products(n, n, mc, pf, pb);
    if (!err) err = cp(D->tC64.pfwd, pf.data(), sizeof(double) * pf.size());
    if (!err) err = cp(D->tC64.pbwd, pb.data(), sizeof(double) * pb.size());
    if (D->tA64.pfwd != nullptr) {
      thomas_chunk_products(n, as, ma, pf, pb);
      if (!err) err = cp(D->tA64.pfwd, pf.data(), sizeof(double) * pf.size());
      if (!err) err = cp(D->tA64.pbwd, pb.data(), sizeof(double) * pb.size());
    }
  }
  if (!err) err = cp(D->tA32.mneg, ma32.data(), sizeof(float) * ma32.size());
  if (L.chain) {  // pivots of the row's sweeps (length nxc); the DST-I tables are the centre's
    D->tR64.plan = D->tC64.plan;
    D->tR32.plan = D->tC32.plan;
    std::vector<double> pr, mr;
    fill_pivots(n, L.cg.nxc, D->delta, desc->kappa, pr);
    mr.resize(pr.size());
    for (size_t i = 0; i < pr.size(); ++i) mr[i] = -D->delta * pr[i];
    std::vector<float> pr32(pr.begin(), pr.end()), mr32(mr.begin(), mr.end());
    if (!err) err = cp(D->tR64.rpiv, pr.data(), sizeof(double) * pr.size());
    if (!err) err = cp(D->tR64.mneg, mr.data(), sizeof(double) * mr.size());
    if (!err) err = cp(D->tR32.rpiv, pr32.data(), sizeof(float) * pr32.size());
    if (!err) err = cp(D->tR32.mneg, mr32.data(), sizeof(float) * mr32.size());
    if (!err) err = cudaStreamSynchronize(D->st);  // the host vectors end with this block
  }
  if (nside) {
    if (!err) err = cp(D->tA64e.rpiv, pae.data(), sizeof(double) * pae.size());
    if (!err) err = cp(D->tA64e.mneg, mae.data(), sizeof(double) * mae.size());
    if (!err) err = cp(D->tA64.plan.W, Wd.data(), sizeof(double) * Wd.size());
    if (!err) err = cp(D->tA64.post, postd.data(), sizeof(double) * postd.size());
  }
  if (!L.chain && fast_solve_cluster_tables(n, D->delta, desc->kappa, cl_sigma, cl_wseed)) {
    if (!err) err = cp(D->tC32.cl_sigma, cl_sigma.data(), sizeof(float) * cl_sigma.size());
    if (!err) err = cp(D->tC32.cl_wseed, cl_wseed.data(), sizeof(float) * cl_wseed.size());
  } else {
    D->tC32.cl_sigma = D->tC32.cl_wseed = nullptr;  // the kernel does not take this length
  }
  LatticeHost lh;
  if (L.lattice) {
    if (!lattice_tables(desc->lattice, n, D->delta, desc->kappa, &lh)) err = cudaErrorInvalidValue;
    if (!err) err = cp(D->lat.nbr, lh.nbr.data(), sizeof(int4) * lh.nbr.size());
    if (!err) err = cp(D->lat.cf, lh.cf.data(), sizeof(int2) * lh.cf.size());
    if (!err) err = cp(D->lat.anb, lh.anb.data(), sizeof(int2) * lh.anb.size());
    if (!err && !lh.faces.empty()) err = cp(D->lat.faces, lh.faces.data(), sizeof(int2) * lh.faces.size());
    if (!err) err = cp(D->lat.gnbr, lh.gnbr.data(), sizeof(int4) * lh.gnbr.size());
    if (!err) err = cp(D->lat.gcn, lh.gcn.data(), sizeof(int) * lh.gcn.size());
    if (!err) err = cp(D->lat.lpiv, lh.lpiv.data(), sizeof(double) * lh.lpiv.size());
  }
  if (!err) err = cp(D->ctab, ct.data(), sizeof(double) * ct.size());
  if (!err && D->gmat != nullptr) {
    // G(j, i) = T(|i-j|) - H(i+j): the same values the table form forms on the fly
    std::vector<double> G((size_t)n * n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) G[(size_t)j * n + i] = ct[i > j ? i - j : j - i] - ct[2 * n + 2 + i + j];
    err = cp(D->gmat, G.data(), sizeof(double) * G.size());
  }
  if (!err) err = cp(D->gsc, gs.data(), sizeof(double) * gs.size());
  if (!err) err = cp(D->arms_dev, arms, sizeof(arms));
  if (!err) err = cudaMemsetAsync(D->f, 0, sizeof(double) * nrhs * L.ntot, D->st);
  if (!err) err = cudaStreamSynchronize(D->st);
  if (!err) err = cudaMallocHost((void**)&D->h_done_pinned, sizeof(int) * (nrhs + 1));
  if (!err) err = cudaEventCreateWithFlags(&D->ev_flags, cudaEventDisableTiming);
  if (err) {
    record_cuda_error(err, "fpg_create_domain");
    if (D->h_done_pinned) cudaFreeHost(D->h_done_pinned);
    delete D;
    return FPG_ECUDA;
  }
  *out = D;
  return FPG_OK;
}

void fpg_destroy_domain(fpg_domain* d) {
  if (!d) return;
  for (auto ev : d->evpool) cudaEventDestroy(ev);
  for (auto ev : d->gev) cudaEventDestroy(ev);
  drop_graph(d);
  if (d->ev_flags) cudaEventDestroy(d->ev_flags);
  if (d->h_done_pinned) cudaFreeHost(d->h_done_pinned);
  delete d;
}

fpg_status fpg_solve_many(fpg_domain* const* doms, int32_t count, double* const* p_dev,
                          fpg_solve_info* const* infos) {
  if (!doms || !p_dev || count < 0) return FPG_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!doms[i] || !p_dev[i]) return FPG_EINVAL;
  std::vector<char> live(count, 1);
  for (int i = 0; i < count; ++i) FPG_TRY(stage_setup(doms[i], p_dev[i]));
  int remaining = count;
  while (remaining > 0) {
    for (int i = 0; i < count; ++i)
      if (live[i]) FPG_TRY(stage_restart(doms[i]));
    for (int i = 0; i < count; ++i) {
      if (!live[i]) continue;
      bool done = false;
      FPG_TRY(stage_poll(doms[i], &done));
      if (done) {
        FPG_TRY(stage_finish(doms[i]));
        bool resume = false;
        FPG_TRY(stage_resume(doms[i], &resume));
        if (!resume) {
          live[i] = 0;
          --remaining;
        }
      } else {
        FPG_TRY(stage_cycle(doms[i]));
      }
    }
  }
  fpg_status all = FPG_OK;
  for (int i = 0; i < count; ++i) {
    const fpg_status s = collect_info(doms[i], infos ? infos[i] : nullptr);
    if (s != FPG_OK && all == FPG_OK) all = s;
  }
  return all;
}

fpg_status fpg_set_rhs(fpg_domain* d, const double* f_dev, int32_t rhs_index) {
  if (!d || !f_dev || rhs_index < -1 || rhs_index >= d->desc.nrhs) return FPG_EINVAL;
  const size_t one = sizeof(double) * d->L.ntot;
  if (rhs_index < 0)
    FPG_CUDA_TRY(cudaMemcpyAsync(d->f, f_dev, one * d->desc.nrhs, cudaMemcpyDeviceToDevice, d->st));
  else
    FPG_CUDA_TRY(cudaMemcpyAsync(d->f + (size_t)rhs_index * d->L.ntot, f_dev, one, cudaMemcpyDeviceToDevice, d->st));
  return FPG_OK;
}

fpg_status fpg_set_rhs_host(fpg_domain* d, const double* f_host, int32_t rhs_index) {
  if (!d || !f_host || rhs_index < -1 || rhs_index >= d->desc.nrhs) return FPG_EINVAL;
  const size_t one = sizeof(double) * d->L.ntot;
  if (rhs_index < 0)
    FPG_CUDA_TRY(cudaMemcpyAsync(d->f, f_host, one * d->desc.nrhs, cudaMemcpyHostToDevice, d->st));
  else
    FPG_CUDA_TRY(cudaMemcpyAsync(d->f + (size_t)rhs_index * d->L.ntot, f_host, one, cudaMemcpyHostToDevice, d->st));
  return FPG_OK;
}

fpg_status fpg_solve(fpg_domain* d, double* p_dev, fpg_solve_info* info) {
  if (!d || !p_dev) return FPG_EINVAL;
  FPG_TRY(solve_launch(d, p_dev));
  return collect_info(d, info);
}

fpg_status fpg_solve_resume(fpg_domain* d, double* p_dev, fpg_solve_info* info) {
  if (!d || !p_dev) return FPG_EINVAL;
  FPG_TRY(solve_launch(d, p_dev, true));
  return collect_info(d, info);
}

fpg_status fpg_solve_async(fpg_domain* d, double* p_dev) {
  if (!d || !p_dev) return FPG_EINVAL;
  return solve_launch(d, p_dev);
}

fpg_status fpg_solve_finish(fpg_domain* d, fpg_solve_info* info) {
  if (!d) return FPG_EINVAL;
  return collect_info(d, info);
}

fpg_status fpg_solve_host(fpg_domain* d, const double* f_host, double* p_host, fpg_solve_info* info) {
  if (!d || !f_host || !p_host) return FPG_EINVAL;
  FPG_TRY(fpg_set_rhs_host(d, f_host, -1));
  FPG_TRY(solve_launch(d, d->pbuf));
  FPG_CUDA_TRY(cudaMemcpyAsync(p_host, d->pbuf, sizeof(double) * d->L.ntot * d->desc.nrhs, cudaMemcpyDeviceToHost,
                               d->st));
  return collect_info(d, info);
}

// ---- operator entry points --------------------------------------------------

fpg_status fpg_apply_precond(fpg_domain* d, const double* v, void* z, int32_t nvec) {
  if (!d || !v || !z || nvec < 0) return FPG_EINVAL;
  const size_t zel = d->prec == 64 ? 8 : 4;
  for (int s = 0; s < nvec; s += d->desc.nrhs) {
    const int c = std::min(d->desc.nrhs, nvec - s);
    FPG_TRY(precond(d, v + (size_t)s * d->L.nc, (char*)z + zel * (size_t)s * d->L.nc, c, nullptr));
  }
  return check_launch();
}

fpg_status fpg_block_solve(fpg_domain* d, int32_t block, const double* v, double* z, int32_t nvec) {
  if (!d || !v || !z || nvec < 0 || block < 0 || block > 4) return FPG_EINVAL;
  const Layout& L = d->L;
  if (L.chain || L.lattice) return FPG_EUNSUPPORTED;
  if (block > 0 && L.ao.off[block - 1] < 0) return FPG_EINVAL;
  const long long len = block == 0 ? L.nc : L.na;
  const LineLayout& LL = block == 0 ? d->LC : (block <= 2 ? d->LWE : d->LSN);
  const FastSolveTables& tb = block == 0 ? d->tC64 : ((L.ao.bc == 1 && (block == 2 || block == 4)) ? d->tA64e : d->tA64);
  const int cap = (int)std::max(1LL, ((long long)d->desc.nrhs * std::max(L.nc, 2 * L.na)) / len);
  for (int s = 0; s < nvec; s += cap) {
    const int c = std::min(cap, nvec - s);
    BatchDesc bd{len, {0, 0, 0, 0}, 1};
    int nl = 0;
    FPG_CUDA_TRY(launch_fast_solve(64, 64, tb, LL, v + (size_t)s * len, bd, z + (size_t)s * len, bd, c,
                                   d->scratch, nullptr, 1, d->st, &nl));
    d->launches += nl;
  }
  return check_launch();
}

fpg_status fpg_apply_schur(fpg_domain* d, const void* z, int32_t zprec, double* w, int32_t nvec) {
  if (!d || !z || !w || nvec < 0 || (zprec != 64 && zprec != 32)) return FPG_EINVAL;
  const size_t zel = zprec == 64 ? 8 : 4;
  for (int s = 0; s < nvec; s += d->desc.nrhs) {
    const int c = std::min(d->desc.nrhs, nvec - s);
    FPG_TRY(schur(d, (const char*)z + zel * (size_t)s * d->L.nc, zprec, w + (size_t)s * d->L.nc, c, nullptr));
  }
  return check_launch();
}

fpg_status fpg_arnoldi_mgs(fpg_domain* d, const double* V, int32_t j, double* w, double* h, int64_t len,
                           int32_t nvec) {
  if (!d || !V || !w || !h || j < 0 || len <= 0 || nvec <= 0 || nvec > d->desc.nrhs) return FPG_EINVAL;
  // v_{j+1} overwrites w: normalise in place; same kernel choice as the solver
  const int csz =
      d->use_cluster ? (d->tune_csz > 0 && len <= 262144 ? d->tune_csz : arnoldi_cluster_size(len)) : 0;
  const int ept = (csz > 0 && d->arnoldi_mode == 1) ? arnoldi_reg_ept(len, csz, d->tune_nt) : 0;
  if (ept > 0) {
    FPG_CUDA_TRY(launch_arnoldi_reg(csz, d->tune_nt, V, (long long)nvec * len, w, nullptr, 64, nullptr, 0, 0.0, 0.0, 0, w, len, j,
                                    nvec, h, 0, j + 2, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
                                    nullptr, nullptr, 0, 0, d->err_dev, d->st));
    d->launches += 1;
  } else if (csz > 0) {
    FPG_CUDA_TRY(launch_arnoldi_cluster(csz, V, (long long)nvec * len, w, w, len, j, nvec, h, 0, j + 2, nullptr,
                                        nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0, 0,
                                        d->st));
    d->launches += 1;
  } else {
    int nl = 0;
    FPG_CUDA_TRY(launch_mgs(V, (long long)nvec * len, w, w, len, j, nvec, d->ks.part, kGmax, h, 0, j + 2, nullptr,
                            pick_gx(len, nvec), d->st, &nl));
    d->launches += nl;
  }
  return check_launch();
}

fpg_status fpg_givens(fpg_domain* d, double* Hcol, double* cs, double* sn, double* g, double* res, int32_t j,
                      int32_t m, int32_t nvec) {
  if (!d || !Hcol || !cs || !sn || !g || !res || j < 0 || j >= m || nvec <= 0) return FPG_EINVAL;
  FPG_CUDA_TRY(launch_givens(Hcol, 0, j + 2, cs, sn, g, res, j, m, nvec, nullptr, nullptr, nullptr, nullptr, 0,
                             d->st));
  d->launches += 1;
  return check_launch();
}

fpg_status fpg_global_residual(fpg_domain* d, const double* f, const double* p, double* out_host, int32_t nvec) {
  if (!d || !f || !p || !out_host || nvec <= 0) return FPG_EINVAL;
  const Layout& L = d->L;
  for (int s = 0; s < nvec; s += d->desc.nrhs) {
    const int c = std::min(d->desc.nrhs, nvec - s);
    FPG_CUDA_TRY(global_apply(d, p + (size_t)s * L.ntot, nullptr, f + (size_t)s * L.ntot, c, d->gres, nullptr, 0.0,
                              nullptr));
    d->launches += 2;
    FPG_CUDA_TRY(cudaMemcpyAsync(out_host + s, d->gres, sizeof(double) * c, cudaMemcpyDeviceToHost, d->st));
    FPG_CUDA_TRY(cudaStreamSynchronize(d->st));
  }
  return FPG_OK;
}

fpg_status fpg_apply_global(fpg_domain* d, const double* p, double* y, int32_t nvec) {
  if (!d || !p || !y || nvec <= 0) return FPG_EINVAL;
  const Layout& L = d->L;
  FPG_CUDA_TRY(global_apply(d, p, y, nullptr, nvec, nullptr, nullptr, 0.0, nullptr));
  d->launches += 1;
  return check_launch();
}

fpg_status fpg_autotune(fpg_domain* d, fpg_tune_result* out) {
  if (!d) return FPG_EINVAL;
  if (d->L.chain || d->L.lattice) return FPG_EUNSUPPORTED;
  drop_graph(d);
  const Layout& L = d->L;
  KrylovState& k = d->ks;
  const int nrhs = d->desc.nrhs, m = d->desc.restart;
  FastSolveTables& tb = d->prec == 64 ? d->tC64 : d->tC32;
  cudaEvent_t e0, e1;
  FPG_CUDA_TRY(cudaEventCreate(&e0));
  FPG_CUDA_TRY(cudaEventCreate(&e1));
  // timing inputs: the first two basis vectors and w (contents do not affect the time)
  FPG_CUDA_TRY(cudaMemsetAsync(k.V, 0, sizeof(double) * (size_t)2 * nrhs * L.nc, d->st));
  FPG_CUDA_TRY(cudaMemsetAsync(k.w, 0, sizeof(double) * (size_t)nrhs * L.nc, d->st));
  // fn returns true when every launch was accepted; a shape whose launch fails
  // (even one the launch consumes the error of) is never chosen
  auto time_it = [&](auto&& fn, int reps) -> float {
    const bool ok = fn();  // warm-up (also sets kernel attributes)
    if (!ok || cudaGetLastError() != cudaSuccess) return 1e30f;
    cudaEventRecord(e0, d->st);
    for (int i = 0; i < reps; ++i) fn();
    cudaEventRecord(e1, d->st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  // a1: line pairs per CTA (generic engine) x warps per CTA of the Thomas kernel
  int best_q = 0, best_mt = 0;
  float best = 1e30f;
  static const int qs[] = {0, 1, 2, 4, 8};  // 0: size-specialised kernels where compiled, else built-in Q
  static const int mts[] = {4, 8};  // the Thomas kernel's launch bound: 8 warps
  for (int q : qs) {
    for (int mt : mts) {
      tb.q = q;
      tb.mt = mt;
      const float t = time_it([&] { return precond(d, k.V, k.Z, nrhs, nullptr) == FPG_OK; }, 3);
      if (t < best) { best = t; best_q = q; best_mt = mt; }
    }
  }
  tb.q = best_q;
  tb.mt = best_mt;
  // a3 (+a4): cluster size (and thread cap) of the fused Arnoldi step, at j = m/2
  int best_c = 0, best_nt = 0;
  float best_a = 1e30f;
  if (d->use_cluster && L.nc <= 262144) {
    const int j = m / 2 < 1 ? 0 : m / 2;
    const int hcol = m + 1, hrhs = m * (m + 1);
    static const int cs_[] = {1, 2, 4, 8, 10, 12, 14, 15, 16};
    static const int nts[] = {256, 512};
    for (int c : cs_) {
      for (int nt : nts) {
        const int ept = d->arnoldi_mode == 1 ? arnoldi_reg_ept(L.nc, c, nt) : 0;
        if (d->arnoldi_mode != 1 && nt != nts[0]) continue;
        const float t = time_it([&] {
          if (ept > 0)
            return launch_arnoldi_reg(c, nt, k.V, (long long)nrhs * L.nc, k.w, nullptr, 64, nullptr, 0, 0.0, 0.0, 0,
                               k.V + (size_t)(j + 1) * nrhs * L.nc, L.nc, j, nrhs, k.H, hcol, hrhs, nullptr, nullptr,
                               nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0, 0, d->err_dev,
                               d->st) == cudaSuccess;
          else
            return launch_arnoldi_cluster(c, k.V, (long long)nrhs * L.nc, k.w, k.V + (size_t)(j + 1) * nrhs * L.nc, L.nc,
                                   j, nrhs, k.H, hcol, hrhs, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
                                   nullptr, nullptr, 0, 0, d->st) == cudaSuccess;
        }, 3);
        if (t < best_a) { best_a = t; best_c = c; best_nt = nt; }
      }
    }
    d->tune_csz = best_c;
    d->tune_nt = best_nt;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out) {
    out->q = best_q;
    out->mt = best_mt;
    out->cluster = best_c;
    out->threads = best_nt;
    out->precond_ms = best;
    out->arnoldi_ms = best_a < 1e29f ? best_a : 0.0;
  }
  return check_launch();
}

fpg_status fpg_set_option(fpg_domain* d, int32_t option, int32_t value) {
  if (!d) return FPG_EINVAL;
  switch (option) {
    case FPG_OPT_ARNOLDI_CLUSTER:
      if (value < 0 || value > 2) return FPG_EINVAL;
      d->use_cluster = value != 0;
      d->arnoldi_mode = value == 2 ? 2 : 1;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_CUDA_GRAPHS:
      d->use_graphs = value != 0;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_FUSED_FASTSOLVE:
      if ((d->L.chain || d->L.lattice) && value) return FPG_EUNSUPPORTED;  // the one-pass kernel takes whole square blocks
      for (auto* t : {&d->tC64, &d->tC32, &d->tA64, &d->tA32, &d->tA64e}) t->fused = value != 0;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_PRECOND:
      if (value < 0 || value > 3) return FPG_EINVAL;
      if ((d->L.chain || d->L.lattice) && value == 2) return FPG_EUNSUPPORTED;  // Jacobi: written for the cross
      if (d->L.lattice && value == 3) return FPG_EUNSUPPORTED;  // a lattice's default is already block diagonal
      if (!d->L.chain && value == 3) return FPG_EUNSUPPORTED;  // the squares of a coupled row: chains only
      d->precond_kind = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_DST_ENGINE:
      if (value < 0 || value > 2) return FPG_EINVAL;
      for (auto* t : {&d->tC64, &d->tC32, &d->tA64, &d->tA32, &d->tA64e}) t->generic = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_DST_BULK:
      if (value < 0 || value > 2) return FPG_EINVAL;
      for (auto* tt : {&d->tC64, &d->tC32, &d->tA64, &d->tA32, &d->tA64e}) tt->bulk = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_DST_PAIRS:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8) return FPG_EINVAL;
      for (auto* t : {&d->tC64, &d->tC32}) t->q = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_THOMAS_WARPS:
      if (value != 0 && value != 4 && value != 8) return FPG_EINVAL;
      for (auto* t : {&d->tC64, &d->tC32}) t->mt = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_CLUSTER_FASTSOLVE:
      if (value < 0 || value > 1) return FPG_EINVAL;
      d->tC32.cluster = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_THOMAS_PRODUCTS:
      if (value < 0 || value > 1) return FPG_EINVAL;
      for (auto* tt : {&d->tC64, &d->tA64}) tt->use_products = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_WAIT_LIMIT:
      if (value < 0) return FPG_EINVAL;
      for (auto* tt : {&d->tC64, &d->tC32, &d->tA64, &d->tA32, &d->tA64e, &d->tR64, &d->tR32}) tt->wait_limit = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_ARM_REFINE:
      if (value < 0 || value > 4) return FPG_EINVAL;
      d->arm_refine = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_SCHUR_TRANSFORM:
      if (value < 0 || value > 2) return FPG_EINVAL;
      d->schur_transform = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_ARNOLDI_CSZ:
      if (value < 0 || value > 16) return FPG_EINVAL;
      d->tune_csz = value;
      drop_graph(d);
      return FPG_OK;
    case FPG_OPT_ARNOLDI_THREADS:
      if (value != 0 && value != 256 && value != 512) return FPG_EINVAL;
      d->tune_nt = value;
      drop_graph(d);
      return FPG_OK;
    default: return FPG_EINVAL;
  }
}

fpg_status fpg_set_profiling(fpg_domain* d, int32_t on) {
  if (!d) return FPG_EINVAL;
  d->profiling = on != 0;
  if (d->profiling && d->evpool.empty()) {
    d->evpool.resize(kMaxEvents);
    for (auto& ev : d->evpool) FPG_CUDA_TRY(cudaEventCreate(&ev));
  }
  for (int i = 0; i < kPhases; ++i) {
    d->phase_ms[i] = 0;
    d->phase_launches[i] = 0;
  }
  return FPG_OK;
}

fpg_status fpg_phase_stats(fpg_domain* d, int32_t phase, int64_t* launches, double* ms) {
  if (!d || phase < 0 || phase >= kPhases) return FPG_EINVAL;
  ev_collect(d);  // events of operator calls made since the last solve
  if (launches) *launches = d->phase_launches[phase];
  if (ms) *ms = d->phase_ms[phase];
  return FPG_OK;
}

fpg_status fpg_set_history(fpg_domain* d, double* dev_buf, int32_t len) {
  if (!d || len < 0 || (len > 0 && !dev_buf)) return FPG_EINVAL;
  d->hist = len > 0 ? dev_buf : nullptr;
  d->hist_len = len;
  drop_graph(d);  // the recording launches join or leave the captured cycle
  return FPG_OK;
}

fpg_status fpg_set_stream(fpg_domain* d, void* stream) {
  if (!d) return FPG_EINVAL;
  d->st = (cudaStream_t)stream;  // an instantiated cycle graph launches on any stream
  return FPG_OK;
}

fpg_status fpg_arnoldi_shape(fpg_domain* d, int32_t* kind, int32_t* cluster, int32_t* threads, int32_t* ctas) {
  if (!d) return FPG_EINVAL;
  const Layout& L = d->L;
  // the same choice as the solver's Arnoldi step
  const int csz = d->use_cluster ? (d->tune_csz > 0 ? d->tune_csz : arnoldi_cluster_size(L.nc)) : 0;
  const int ept = (csz > 0 && d->arnoldi_mode == 1 && !L.chain && !L.lattice) ? arnoldi_reg_ept(L.nc, csz, d->tune_nt)
                                                                                 : 0;
  int k = 0, t = 256;
  if (ept > 0) {
    k = 1;
    t = arnoldi_reg_threads(L.nc, csz, ept);
  } else if (csz > 0) {
    k = 2;
  }
  if (kind) *kind = k;
  if (cluster) *cluster = k ? csz : 0;
  if (threads) *threads = t;
  if (ctas) *ctas = k ? csz * d->desc.nrhs : 0;
  return FPG_OK;
}

fpg_status fpg_fast_solve_path(fpg_domain* d, int32_t* path) {
  if (!d || !path) return FPG_EINVAL;
  if (d->L.chain && d->precond_kind != 1) {  // the row solve, or the squares (same engine choice)
    *path = d->precond_kind == 0 ? fast_solve_path(d->prec, d->prec == 64 ? d->tR64 : d->tR32, d->LR, d->desc.nrhs)
                                 : fast_solve_path(d->prec, d->prec == 64 ? d->tA64 : d->tA32, d->LC1, d->desc.nrhs);
    return FPG_OK;
  }
  if (d->precond_kind != 0) {
    *path = 4;
    return FPG_OK;
  }
  const FastSolveTables& tb = d->prec == 64 ? d->tC64 : d->tC32;
  *path = fast_solve_path(d->prec, tb, d->LC, d->desc.nrhs);
  return FPG_OK;
}

fpg_status fpg_launch_count(fpg_domain* d, int64_t* launches) {
  if (!d || !launches) return FPG_EINVAL;
  *launches = d->launches;
  return FPG_OK;
}

fpg_status fpg_probe_fma_peak(int32_t precision, double* flops) {
  if (!flops || (precision != 64 && precision != 32)) return FPG_EINVAL;
  int dev = 0, sms = 0;
  FPG_CUDA_TRY(cudaGetDevice(&dev));
  FPG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st;
  FPG_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  const int iters = precision == 64 ? 256 : 8192;
  launch_fma_probe(precision, blocks, 16, st);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    launch_fma_probe(precision, blocks, iters, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (err != cudaSuccess) {
    record_cuda_error(err, "fma probe");
    return FPG_ECUDA;
  }
  // 256 threads x 8 chains x 8 unrolled FMAs x iters, 2 flops each
  *flops = 2.0 * blocks * 256.0 * 64.0 * iters / (best * 1e-3);
  return FPG_OK;
}

}  // extern "C"
