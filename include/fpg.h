/*
 * fpg.h -- C ABI of the GB300 FFT-preconditioned Schur-complement GMRES solver
 * for the discrete 5-point Helmholtz-Poisson equation on block domains.
 *
 * Problem (Eq. 1 with the central differences of Eq. "Poisson_central"):
 *     (p[i+1,j] + p[i-1,j] + p[i,j+1] + p[i,j-1] - 4 p[i,j]) / h^2 + kappa p[i,j] = f[i,j]
 * on the L, T or cross domain built from unit squares (Sec. 2.3, Sec. 3), one
 * grid size n per domain, h = 1/(n+1), zero Dirichlet data on the outer edge.
 *
 * Method (Sec. 2.3-2.4, Alg. "fft_dd_solver"): the arms are "independent"
 * blocks and the centre C is the one "coupled" block.  The arms are eliminated
 * exactly (Eq. "Schur_subeq"), the Schur system L_c p_c = f'_c of the centre is
 * solved by GMRES with the paper's preconditioner A_c^{-1} applied on the right
 * (flexible GMRES), each application being one fast solve (DST-I along x,
 * Thomas along y per mode, inverse DST-I; Eqs. "eigen_trans"-"trans_subeq"), and
 * the arms are recovered by back substitution.
 *
 * Vector layout (all FP64 unless stated; "block order"):
 *   the centre C (n x n nodes (i h, j h), i,j = 1..n), then the arms present in
 *   the order W, E, S, N (cross = C,W,E,S,N; T = C,W,E,S; L = C,E,N).  Each arm
 *   owns the grid line it shares with C: W and E hold (n+1) x n nodes, S and N
 *   hold n x (n+1).  Inside a block: row-major, x fastest.  Several right-hand
 *   sides are stored one full vector after another.
 *
 * Chain of K crosses (geometry = FPG_GEOM_CHAIN, desc.chain = K, 2 <= K <= 5;
 * several coupled blocks, Sec. 2.3-2.4): 2K - 1 unit squares in a row along x
 * (centres at even positions, links between them) are the coupled set, solved
 * together by flexible GMRES preconditioned with the row's own operator (one
 * fast solve of the whole row; FPG_OPT_PRECOND = 3: the block diagonal of its
 * squares, one fast solve each); arms W and E at the row's ends and S_i, N_i
 * below and above centre i are eliminated exactly.  Vector layout: the row as
 * one rectangle of nx_c = (2K-1)(n+1) - 1 columns by n rows (x fastest; each
 * square owns the line it shares with the next), then W, E ((n+1) x n), S_1..S_K,
 * N_1..N_K (n x (n+1)); centre i's columns start at 2 i (n+1).  Reduced Schur
 * form, Dirichlet edges, A_c^{-1} or identity preconditioner only (else
 * FPG_EUNSUPPORTED); fpg_block_solve and fpg_autotune are not offered.
 *
 * General concatenated geometry (geometry = FPG_GEOM_LATTICE; Sec. 2.3-2.4 and
 * the rule after Alg. "fft_dd_solver": a sub-domain adjacent to only one other
 * is independent, the others are coupled): any edge-connected set of 2..64 unit
 * squares [i, i+1] x [j, j+1], 0 <= i, j < 8, given as desc.lattice with bit
 * i + 8 j set.  A square with one edge neighbour is independent, eliminated
 * exactly, and owns the grid line it shares with that neighbour; squares with
 * two or more neighbours are coupled (of two squares, the first is taken as
 * coupled).  The coupled set -- the coupled squares' n x n interiors, every grid
 * line shared by two coupled squares (a link, n points) and every lattice
 * vertex with four squares around it (a junction, one point) -- is solved by
 * flexible GMRES preconditioned with the block diagonal of its parts (a fast
 * solve per coupled square, a tridiagonal solve per link, the diagonal of each
 * junction).  Vector layout: the coupled set first -- coupled squares in bit
 * order (n x n), the links across vertical edges then across horizontal edges,
 * each ordered by (j, i) of the left or lower square (n points along the line),
 * the junctions ordered by the vertex's (Y, X) -- then the independent squares
 * in bit order, (n+1) x n when the neighbour is west or east, n x (n+1) when it
 * is south or north, the shared line first (neighbour west or south) or last
 * (east or north); x fastest in every block.  At most 8 independent squares
 * with a west or east neighbour and 8 with a south or north one; reduced Schur
 * form, Dirichlet edges, block-diagonal or identity preconditioner
 * (FPG_OPT_PRECOND 0 or 1); fpg_block_solve and fpg_autotune are not offered
 * (else FPG_EUNSUPPORTED; a mask that is not edge-connected is FPG_EINVAL).
 *
 * Neumann-sided cross (boundary = FPG_BC_NEUMANN_SIDES; the boundary pattern
 * of the paper's precision validation, Sec. 3.1 Eq. "cross_equation"): zero
 * Dirichlet at the four far ends of the arms, zero normal derivative on the
 * arms' sides.  The grid is cell-centred, h = 1/n, an unknown at every cell
 * centre ((I + 1/2) h, (J + 1/2) h); every block, arms included, is n x n, in
 * the same block order.  The Neumann faces use the matrix of Eq.
 * "submat_Neumann" (the row loses one delta); a Dirichlet face half a cell away
 * makes the row gain -delta.  The arms' fast solves run DCT-II lines along
 * their interface (Sec. 2.2) instead of DST-I; the centre keeps DST-I.
 *
 * Memory: the library never allocates device memory on the solve path.  The
 * caller passes one device workspace (size from fpg_workspace_bytes) at
 * creation and owns it; the handle itself is host memory owned by the library.
 * All device work is ordered on the stream given at creation; functions that
 * return host results synchronise that stream.
 *
 * Errors: every call returns an fpg_status; no C++ exception crosses the ABI.
 * Device waits are bounded (FPG_OPT_WAIT_LIMIT): a wait that gives up makes the
 * solve return FPG_ETIMEOUT, and the stream and context stay usable.
 */
#ifndef FPG_H
#define FPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FPG_OK = 0,
  FPG_EINVAL = 1,       /* bad argument or descriptor */
  FPG_ENOMEM = 2,       /* workspace smaller than fpg_workspace_bytes() */
  FPG_ECUDA = 3,        /* a CUDA call failed; see fpg_last_cuda_error() */
  FPG_ENOCONV = 4,      /* max_iters reached: p holds the last iterate */
  FPG_ETIMEOUT = 5,     /* a bounded device wait gave up */
  FPG_EUNSUPPORTED = 6, /* valid request this build does not provide */
  FPG_EBUDGET = 7       /* admission refused: over the memory budget */
} fpg_status;

typedef enum {
  FPG_GEOM_L = 0,
  FPG_GEOM_T = 1,
  FPG_GEOM_CROSS = 2,
  FPG_GEOM_CHAIN = 3,
  FPG_GEOM_LATTICE = 4
} fpg_geometry;

typedef enum {
  FPG_BC_DIRICHLET = 0,     /* every outer edge Dirichlet; vertex-centred grid, h = 1/(n+1) */
  FPG_BC_NEUMANN_SIDES = 1  /* cross only: Neumann arm sides, Dirichlet far ends; cell-centred, h = 1/n;
                               n even with prime factors <= 13, n <= 2048 (else FPG_EUNSUPPORTED) */
} fpg_boundary;

typedef enum {
  FPG_SCHUR_REDUCED = 0, /* arm response by its exact interface table (DST, x g_k, DST) */
  FPG_SCHUR_LITERAL = 1  /* arm response by a full fast solve of every arm (Eq. "precond_basis_equ") */
} fpg_schur_mode;

typedef struct {
  int32_t geometry;          /* fpg_geometry */
  int32_t n;                 /* interior points per side of the centre block, 2 <= n <= 4096 */
  double kappa;              /* Helmholtz shift, kappa <= 0 */
  int32_t nrhs;              /* right-hand sides solved together, >= 1 */
  int32_t restart;           /* GMRES restart length m, 1..128 */
  double rtol;               /* stop when ||f - K p||_2 <= rtol ||f||_2 (global vectors) */
  int32_t max_iters;         /* cap on total GMRES steps per right-hand side */
  int32_t precond_precision; /* 64: FP64 fast solve; 32: FP32 fast solve (FP64 outer loop) */
  int32_t schur_mode;        /* fpg_schur_mode */
  int32_t boundary;          /* fpg_boundary (0 = all Dirichlet) */
  int32_t chain;             /* FPG_GEOM_CHAIN: number of crosses K, 2..5; other geometries: 0 */
  uint64_t lattice;          /* FPG_GEOM_LATTICE: the squares, bit i + 8 j; other geometries: 0 */
} fpg_domain_desc;

typedef struct {
  int32_t iterations;   /* GMRES steps taken */
  int32_t restarts;     /* restart cycles run */
  int32_t status;       /* fpg_status of this right-hand side */
  int32_t reserved;
  double residual;      /* final ||f - K p||_2 / ||f||_2, computed on the device */
  double schur_residual;/* final GMRES estimate |g_{j+1}| / ||f||_2 */
} fpg_solve_info;

typedef struct fpg_domain fpg_domain;

/* Human-readable name of a status code (static storage). */
const char* fpg_status_string(fpg_status s);
/* Text of the last CUDA error this thread saw (static storage). */
const char* fpg_last_cuda_error(void);
/* Library version string. */
const char* fpg_version(void);

/* Number of unknowns of one right-hand side: n^2 + arms * n (n+1); 5 n^2 for
 * the Neumann-sided cross; nx_c n + (2K + 2) n (n+1) for a chain. */
fpg_status fpg_unknowns(const fpg_domain_desc* desc, int64_t* count);

/* Device workspace needed by fpg_create_domain for this descriptor (bytes).
 * Pure host computation; allocates nothing. */
fpg_status fpg_workspace_bytes(const fpg_domain_desc* desc, size_t* bytes);

/* Build a domain: host tables (eigenvalues, Thomas pivots, DST twiddles,
 * interface table g_k) computed in FP64 and copied into the caller's
 * workspace on `stream` (a cudaStream_t, NULL = legacy default stream).
 * dev_workspace must stay valid until fpg_destroy_domain.
 * Errors: FPG_EINVAL (descriptor), FPG_ENOMEM (bytes too small), FPG_ECUDA. */
fpg_status fpg_create_domain(const fpg_domain_desc* desc, void* dev_workspace, size_t bytes,
                             void* stream, fpg_domain** out);

/* Copy right-hand side(s) into the domain (stream-ordered device-to-device copy).
 * f_dev: device pointer, block order; rhs_index = -1 copies all nrhs vectors
 * (nrhs * unknowns doubles), otherwise one vector into slot rhs_index.
 * The caller may reuse f_dev once the stream has passed this point. */
fpg_status fpg_set_rhs(fpg_domain* d, const double* f_dev, int32_t rhs_index);

/* Same as fpg_set_rhs from HOST memory (pinned for best speed): one
 * host-to-device copy on the domain's stream. */
fpg_status fpg_set_rhs_host(fpg_domain* d, const double* f_host, int32_t rhs_index);

/* Solve K p = f for every right-hand side (Alg. "fft_dd_solver").
 * p_dev: caller-owned device buffer of nrhs * unknowns doubles (block order).
 * info_host: nrhs entries (may be NULL).  Synchronises the stream.
 * Returns FPG_OK when every right-hand side met rtol, FPG_ENOCONV when some did
 * not (their p holds the last iterate), FPG_ETIMEOUT or FPG_ECUDA. */
fpg_status fpg_solve(fpg_domain* d, double* p_dev, fpg_solve_info* info_host);

/* Launch the solve without waiting (graph-friendly form of fpg_solve): the
 * result and the per-RHS info land on the stream; call fpg_solve_finish to
 * wait and read the info.  Restart decisions are taken on the device. */
fpg_status fpg_solve_async(fpg_domain* d, double* p_dev);
fpg_status fpg_solve_finish(fpg_domain* d, fpg_solve_info* info_host);

/* Checkpoint / resume: solve the domain's right-hand sides starting from the
 * iterates already in p_dev (same layout as fpg_solve's output, e.g. the p of a
 * solve that stopped with FPG_ENOCONV at max_iters, copied out and back).  The
 * residual r = f - K p is formed on the device, the same algorithm runs on r
 * (a right-hand side already at or below rtol gets r = 0 and keeps its p), and
 * the correction is added to p; the acceptance loop then runs as in fpg_solve.
 * info counts the iterations of this call only.  A right-hand side f = 0 with a
 * nonzero p runs to max_iters (its rtol ||f|| is 0).  Same errors as fpg_solve. */
fpg_status fpg_solve_resume(fpg_domain* d, double* p_dev, fpg_solve_info* info_host);

/* End-to-end convenience: host f -> device -> solve -> host p (both pinned for
 * best speed), all on the domain's stream. */
fpg_status fpg_solve_host(fpg_domain* d, const double* f_host, double* p_host,
                          fpg_solve_info* info_host);

void fpg_destroy_domain(fpg_domain* d);

/* Solve several domains together -- mixed geometries, sizes, kappas and
 * precisions (the batching form of Alg. "fft_dd_solver").  Each domain's work is
 * issued on the stream it was created with; their restart cycles are
 * interleaved from this one host thread, so the kernels of different domains
 * overlap on the GPU when their streams differ.  p_dev[i]: solution buffer of
 * domain i (its right-hand sides set with fpg_set_rhs); infos[i]: nrhs_i
 * entries or NULL (infos itself may be NULL).  Returns FPG_OK when every
 * right-hand side of every domain met its rtol, else the first other status. */
fpg_status fpg_solve_many(fpg_domain* const* doms, int32_t count, double* const* p_dev,
                          fpg_solve_info* const* infos);

/* ---- batch runtime: continuous batching of requests (serving) --------------
 * A batch holds resident domains carved from one caller-owned device pool.  A
 * request is a domain descriptor whose nrhs (1..slots) counts the request's
 * right-hand sides, plus device pointers to them (f, block order, nrhs full
 * vectors) and to its solution buffer (p, same shape).  Requests with equal
 * descriptors apart from nrhs form one queue, served by resident domains of
 * that descriptor with `slots` right-hand sides each: an idle domain takes the
 * oldest queued requests whose right-hand sides fit and solves them as one
 * batch (unused slots carry zero); while all of a descriptor's domains are
 * busy and requests wait, another domain of it is created if the pool has
 * room without evicting (up to max_per_key).  Every resident domain runs on its own CUDA stream
 * created by the library, so batches overlap on the device.  Admission needs
 * one domain of the descriptor (workspace + solution buffer,
 * fpg_workspace_bytes + 8 slots unknowns bytes); when the pool or max_domains
 * is short, idle domains of descriptors with empty queues are evicted least
 * recently used first, and a request that still finds no domain is refused
 * with FPG_EBUDGET and nothing is queued.
 * fpg_batch_step never waits on the device: it advances every domain whose
 * last enqueued stage finished (restart flags, acceptance check, copy-out) and
 * starts idle domains; *completed = tickets finished in this step, the first
 * min(*completed, cap) of them written to finished_tickets (host array, may be
 * NULL when cap = 0; the others stay pollable).  The caller
 * drives admit / step / poll from one host thread.  f must hold its values
 * before fpg_batch_admit returns (synchronise the producing stream); f and p
 * stay owned by the caller and must stay valid until fpg_batch_poll reports
 * the ticket done (done = 1 also releases the ticket; info, if not NULL,
 * receives nrhs entries).  fpg_batch_destroy waits for the device and frees
 * every resident domain; the pool itself stays the caller's.
 * Errors: FPG_EINVAL (arguments, descriptor, unknown ticket), FPG_EBUDGET,
 * FPG_EUNSUPPORTED (descriptor), FPG_ENOMEM, FPG_ECUDA. */
typedef struct {
  int32_t slots;       /* right-hand sides per resident domain, 1..64 */
  int32_t max_domains; /* resident domains at most, 1..256 */
  int32_t max_per_key; /* resident domains per descriptor, 1..16 (0: 4) */
  int32_t max_busy;    /* domains solving at once, >= 1 (0: no limit); batches start oldest request first */
} fpg_batch_desc;

typedef struct {
  int32_t resident;     /* resident domains */
  int32_t busy;         /* of them solving or copying out */
  int32_t queued;       /* requests waiting for their domain's next batch */
  int32_t open_tickets; /* admitted requests not yet finished */
  int64_t pool_used;    /* pool bytes held by resident domains */
  int64_t created;      /* domains created so far */
  int64_t evicted;      /* domains evicted so far */
} fpg_batch_stats_t;

typedef struct fpg_batch fpg_batch;
fpg_status fpg_batch_create(const fpg_batch_desc* desc, void* dev_pool, size_t pool_bytes, fpg_batch** out);
fpg_status fpg_batch_admit(fpg_batch* b, const fpg_domain_desc* request, const double* f_dev, double* p_dev,
                           int64_t* ticket);
fpg_status fpg_batch_step(fpg_batch* b, int64_t* finished_tickets, int32_t cap, int32_t* completed);
fpg_status fpg_batch_poll(fpg_batch* b, int64_t ticket, int32_t* done, fpg_solve_info* info);
fpg_status fpg_batch_stats(fpg_batch* b, fpg_batch_stats_t* out);
void fpg_batch_destroy(fpg_batch* b);

/* ---- operator entry points: each hot-path step on its own ------------------ */

/* a1: preconditioner apply z = A_c^{-1} v for nvec centre-block vectors
 * (n*n doubles each).  z is FP64 for precond_precision 64, FP32 for 32.
 * One fast solve per vector (DST-I along x, Thomas along y, inverse DST-I;
 * Eqs. "eigen_trans"-"trans_subeq"). */
fpg_status fpg_apply_precond(fpg_domain* d, const double* v_dev, void* z_dev, int32_t nvec);

/* Fast solve on one kind of block for nvec vectors: block 0 = centre C,
 * 1..4 = arm W, E, S, N (the arm must exist in the geometry).  FP64 in/out. */
fpg_status fpg_block_solve(fpg_domain* d, int32_t block, const double* v_dev, double* z_dev,
                           int32_t nvec);

/* a2: Schur matvec w = L_c z = A_c z - sum_a R_ca A_a^{-1} R_ac z (Eq.
 * "Schur_subeq") for nvec centre vectors.  z_prec = 64 (double) or 32 (float). */
fpg_status fpg_apply_schur(fpg_domain* d, const void* z_dev, int32_t z_prec, double* w_dev,
                           int32_t nvec);

/* a3: one Arnoldi step by modified Gram-Schmidt for nvec independent systems.
 * V_dev: (j+1) basis vectors per system, layout [j+1][nvec][len]; w_dev: [nvec][len],
 * overwritten by v_{j+1}; h_dev: [nvec][j+2] doubles receives h_{0..j} and h_{j+1,j}. */
fpg_status fpg_arnoldi_mgs(fpg_domain* d, const double* V_dev, int32_t j, double* w_dev,
                           double* h_dev, int64_t len, int32_t nvec);

/* a4: Givens step on column j of Hbar for nvec systems (device arrays):
 * Hcol [nvec][j+2] (in/out), cs, sn [nvec][m], g [nvec][m+1] (in/out).
 * res_dev [nvec] receives |g_{j+1}|. */
fpg_status fpg_givens(fpg_domain* d, double* Hcol_dev, double* cs_dev, double* sn_dev,
                      double* g_dev, double* res_dev, int32_t j, int32_t m, int32_t nvec);

/* a7: global relative residual ||f - K p||_2 / ||f||_2 for nvec full vectors;
 * out_host receives nvec doubles.  Synchronises. */
fpg_status fpg_global_residual(fpg_domain* d, const double* f_dev, const double* p_dev,
                               double* out_host, int32_t nvec);

/* Global operator y = K p for nvec full vectors (block order). */
fpg_status fpg_apply_global(fpg_domain* d, const double* p_dev, double* y_dev, int32_t nvec);

/* ---- fast solve without allocation ---------------------------------------------
 *
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc and cannot hand fpg_create_domain a workspace -- code
 * running inside another framework's memory pool, on a path whose device memory
 * was fixed in advance, or in a context where allocating would stall or fail.
 *
 * fpg_fast_solve_noalloc computes z = A^{-1} v, the fast solve of the centre
 * block, for nvec n x n Dirichlet squares (spacing h = 1/(n+1), shift kappa,
 * each v and z n*n doubles, row-major), with the library's fast-solve kernels.
 * Its scratch (spectral coefficients and the DST / Thomas tables) is one
 * file-scope device array of about 20 MiB that every GPU loading the library
 * holds until the process exits; no device or host memory is allocated.
 *   - Limits: 2 <= n <= FPG_NOALLOC_MAX_N, 1 <= nvec <= FPG_NOALLOC_MAX_NVEC,
 *     nvec * n * n <= FPG_NOALLOC_MAX_POINTS, kappa <= 0.  Anything beyond
 *     returns FPG_EINVAL, the reason readable from fpg_last_cuda_error().
 *   - The first call on a device performs that device's set-up (it looks up
 *     the array's device address); make that first call before any stream
 *     capture.  A call whose (n, kappa) differs from the previous call's
 *     rebuilds the tables on the host, copies them on `stream` and waits for
 *     that stream.
 *   - Every call shares the one array and leaves its contents behind: calls
 *     that overlap on the GPU (other streams, other threads) race.
 * v_dev, z_dev: device pointers owned by the caller; stream: a cudaStream_t. */
#define FPG_NOALLOC_MAX_N 512
#define FPG_NOALLOC_MAX_POINTS (1LL << 21)
#define FPG_NOALLOC_MAX_NVEC 4096
fpg_status fpg_fast_solve_noalloc(int32_t n, double kappa, const double* v_dev, double* z_dev,
                                  int32_t nvec, void* stream);

/* ---- options --------------------------------------------------------------- */

typedef enum {
  /* 1 (default): run each Arnoldi step (a3) and its Givens step (a4) as one
   * launch, one thread-block cluster per right-hand side, for centre blocks of
   * up to 262144 unknowns; when a CTA's slice fits in registers the launch also
   * forms the Schur matvec's stencil (a2).  2: the cluster launch without the
   * register-resident form.  0: one launch per modified Gram-Schmidt step. */
  FPG_OPT_ARNOLDI_CLUSTER = 1,
  /* 1 (default): capture one restart cycle (the m Arnoldi steps) into a CUDA
   * graph at the first solve and replay it for every later cycle; 0: launch
   * every kernel from the host.  Not used while profiling is on or when the
   * domain was created on the legacy default stream. */
  FPG_OPT_CUDA_GRAPHS = 2,
  /* Right preconditioner of the Schur iteration (Sec. 3.2):
   * 0 (default): A_c^{-1}, the paper's FFT preconditioner (a1); on a chain the
   *    coupled row's own operator (couplings between its squares included),
   *    inverted by one fast solve of the whole row;
   * 1: none (P = I);  2: Jacobi, the inverse diagonal of L_c (not on chains);
   * 3: chains only -- the block diagonal of the coupled squares' own
   *    operators, one fast solve per square.
   * With 1 or 2 the flexible basis is still stored in the domain's
   * precond_precision. */
  FPG_OPT_PRECOND = 3,
  /* 1: the fast solve (a1, and the arm solves) runs as one kernel per batch --
   * one thread-block cluster per block, the block's spectral coefficients kept
   * in the cluster's shared memory, v read once and z written once -- when the
   * block fits (n <= 512 in FP64 or FP32).  0 (default; faster on GB300 at the
   * sizes measured so far) and larger blocks: three kernels (DST, Thomas,
   * inverse DST) through a scratch array. */
  FPG_OPT_FUSED_FASTSOLVE = 4,
  /* CTAs per right-hand side of the fused Arnoldi step, 1..16 (0: built-in
   * choice or the autotuner's).  The built-in choice for centre vectors of more
   * than 262144 points is the multi-launch MGS; a value here runs the cluster
   * kernel (w in HBM) for them instead. */
  FPG_OPT_ARNOLDI_CSZ = 5,
  /* Thread cap per CTA of the register-resident Arnoldi kernel: 256 or 512
   * (0: 256 when the centre slice of one CTA fits, else 512). */
  FPG_OPT_ARNOLDI_THREADS = 6,
  /* DST kernels of the fast solve: 0 (default) the size-specialised line DST
   * where one is compiled for the length and pays off (see
   * fpg_fast_solve_path), 1 always the generic FFT engine, 2 the specialised
   * kernels wherever one is compiled. */
  FPG_OPT_DST_ENGINE = 7,
  /* Reduced Schur term (FPG_SCHUR_REDUCED) of the cross, T and L: 0 (default)
   * as the product of the interface lines with the stored n x n matrix
   * G(i, j) = T(|i-j|) - H(i+j) (all arms of a right-hand side per CTA: one
   * FMA per element of G and arm); 1 as delta^2 Q diag(g_k) Q with two DST-I per
   * interface line where the size-specialised DST is compiled (n = 64, 256,
   * 512) -- fewer operations, but only (lines / line batch) CTAs; 2 as the
   * Toeplitz-minus-Hankel sum c(|i-j|) - c(i+j+2) formed on the fly, one thread
   * per output and arm.  Same operator; the forms differ only in rounding. */
  FPG_OPT_SCHUR_TRANSFORM = 8,
  /* Iterative-refinement steps (0..4, default 1) of every arm solve in the
   * setup (q_a = A_a^{-1} f_a) and the finish (p_a = A_a^{-1}(f_a - R_ac p_c)):
   * each step is out += A_a^{-1}(in - A_a out) in FP64. */
  FPG_OPT_ARM_REFINE = 9,
  /* Form of the FP32 forward DST of the size-specialised path for blocks with
   * contiguous, 16-byte aligned rows.  0 (default): where n + 1 is 513 or
   * 1025 and the sweep length is a whole number of tiles, a persistent
   * streaming kernel (two CTAs per SM; the next tile's FP64 rows arrive by a
   * bulk asynchronous copy, cp.async.bulk on an mbarrier, while the current one
   * is transformed in place), else one CTA per tile.  1: a persistent kernel
   * with one CTA per SM and the per-tile engine's buffers.  2: one CTA per tile.
   * All three give bit-identical results. */
  FPG_OPT_DST_BULK = 10,
  /* Tries of every bounded device wait (default 2^22, each try a
   * hardware-suspended mbarrier test; 0: give up at once).  A wait that runs
   * out records it in the domain's status word, the kernel that waited lets its
   * copy in flight land and returns, and the solve reports FPG_ETIMEOUT for
   * every right-hand side.  The waits this option bounds are the bulk-copy
   * waits of FPG_OPT_DST_BULK's persistent kernels (forms 0 and 1).  The Arnoldi step's
   * exchange of projection partials between the CTAs of a cluster waits on an
   * mbarrier too, with a fixed limit of 2^22 tries that only a stopped CTA can
   * reach (its protocol cannot continue after an early give-up); reaching it
   * also sets the status word and gives FPG_ETIMEOUT. */
  FPG_OPT_WAIT_LIMIT = 11,
  /* 1: the FP32 preconditioner (a1 with precond_precision = 32) of centre
   * blocks with n = 64 or 512 runs as one kernel per batch: one thread-block
   * cluster per block (n / 32 CTAs of 32 lines each), the block's spectral
   * coefficients kept in the cluster's shared memory, the tridiagonal sweeps
   * carried across the CTAs through distributed shared memory, v read once
   * and z written once.  0: the three-kernel path.  Other lengths, FP64 and
   * blocks that are not 16-byte aligned always take the other paths. */
  FPG_OPT_CLUSTER_FASTSOLVE = 12,
  /* Launch shapes of the centre's fast solve, as fpg_autotune sets them: line
   * pairs per CTA of the generic FFT engine (0: the size-specialised kernels
   * where compiled, else the built-in choice; 1, 2, 4 or 8), and warps (modes)
   * per CTA of the Thomas kernel (0: 8; 4 or 8). */
  FPG_OPT_DST_PAIRS = 13,
  FPG_OPT_THOMAS_WARPS = 14,
  /* 1 (default): the FP64 Thomas sweeps of the centre and the Dirichlet arms read
   * the carries' running products of the multipliers (-delta r_s inside each lane's
   * chunk of rows) from tables built with the domain, multiplied on the host in the
   * kernel's own order: four FP64 multiplications per row fewer, bit-identical
   * results.  0: the kernel forms them itself. */
  FPG_OPT_THOMAS_PRODUCTS = 15
} fpg_option;

/* Move a domain to another CUDA stream (a cudaStream_t; NULL = the default
 * stream) for its later calls, e.g. a serving worker that reuses resident
 * domains on its own stream.  The caller orders the switch: work the domain
 * issued on its previous stream must be complete or ordered before the next
 * call.  A domain must never be used from two streams at once. */
fpg_status fpg_set_stream(fpg_domain* d, void* stream);

/* Set an option on a domain (affects later calls).  FPG_EINVAL if unknown. */
fpg_status fpg_set_option(fpg_domain* d, int32_t option, int32_t value);

/* ---- autotuning ------------------------------------------------------------- */

typedef struct {
  int32_t q;         /* line pairs per CTA in the DST kernels of a1 */
  int32_t mt;        /* modes (one warp each) per CTA in the Thomas kernel of a1 */
  int32_t cluster;   /* CTAs per right-hand side in the fused Arnoldi step (0: not tuned) */
  int32_t threads;   /* thread cap per CTA of that step (256 or 512; 0: not tuned) */
  double precond_ms; /* time of one preconditioner application (all nrhs vectors) at the choice */
  double arnoldi_ms; /* time of one Arnoldi step at j = m/2 at the choice */
} fpg_tune_result;

/* Time the launch shapes of the hot kernels on this domain's own buffers
 * (precision, n, nrhs as created) and keep the fastest: the line batch (q) and
 * Thomas CTA width (mt) of the fast solve, the cluster size and CTA width of the
 * Arnoldi step.
 * Overwrites the domain's Krylov buffers (call it between solves).  The
 * choices stay with the domain; out (may be NULL) reports them. */
fpg_status fpg_autotune(fpg_domain* d, fpg_tune_result* out);

/* ---- measurement ----------------------------------------------------------- */

/* Residual history (the residual curves of the GMRES study, Sec. 3.2): with a
 * caller-owned device buffer of nrhs x len doubles, every Arnoldi step of later
 * solves writes the GMRES residual estimate |g_{j+1}| of the Schur system of each
 * right-hand side to buf[r * len + i], i = that right-hand side's step count - 1
 * (i < len; relative values: divide by ||f||_2).  Entries past the last step are
 * left untouched.  len = 0 (buf may be NULL) stops recording; the buffer must
 * stay valid until then or until the domain is destroyed.  One small extra
 * launch per Arnoldi step while recording.  Errors: FPG_EINVAL. */
fpg_status fpg_set_history(fpg_domain* d, double* dev_buf, int32_t len);

/* Kernel-level timing of the last fpg_solve on this domain: launches issued and
 * the device time (ms, CUDA events on the domain stream) of each phase.
 * phase: 0 = preconditioner (a1), 1 = Schur matvec (a2), 2 = Arnoldi (a3),
 * 3 = Givens (a4), 4 = cycle end (a5), 5 = setup/finish (a6), 6 = residual (a7);
 * 7, 8, 9 = the three kernels of a1 on their own (forward DST, Thomas, inverse DST);
 * 10 = the fused one-pass fast-solve kernel of a1.
 * Timing is only collected when enabled with fpg_set_profiling(d, 1). */
fpg_status fpg_set_profiling(fpg_domain* d, int32_t on);
fpg_status fpg_phase_stats(fpg_domain* d, int32_t phase, int64_t* launches, double* ms);
/* Total kernel launches issued by the library on this domain so far. */
fpg_status fpg_launch_count(fpg_domain* d, int64_t* launches);

/* ---- rectangle fast solves (Sec. 2.1-2.2) ----------------------------------
 * z = A^{-1} v for nvec rectangles of n_t x n_s points (row-major, t fastest,
 * FP64, device pointers; v and z may not alias), spacing h both ways
 * (delta = 1/h^2), kappa <= 0 on the diagonal, homogeneous Dirichlet ends along
 * s (vertex-centred: the zero neighbours sit one step beyond rows 0 and n_s-1).
 * Along t, by kind:
 *   FPG_RECT_DIRICHLET: zero neighbours one step beyond both ends; DST-I
 *     (Eq. "Dirichlet_mat_decomp"), eigenvalues -4 delta sin^2(k pi/(2(n_t+1))),
 *     k = 1..n_t; 2 <= n_t <= 4096 (the solver's own engine: any length).
 *   FPG_RECT_NEUMANN (Eq. "submat_Neumann"): zero normal derivative half a step
 *     beyond both ends (the first and last rows lose one delta: cell-centred
 *     points); DCT-II, basis cos(k pi (j-1/2)/n_t), eigenvalues
 *     -4 delta sin^2(k pi/(2 n_t)), k = 0..n_t-1; n_t even, 2 <= n_t <= 2048.
 *   FPG_RECT_PERIODIC (Eq. "submat_Periodic"): t wraps around (circulant);
 *     real modes = Re and Im of each line's DFT (mode m: Re X_m for 2m <= n_t,
 *     Im X_m otherwise), eigenvalues -4 delta sin^2(pi m/n_t); 2 <= n_t <= 2048.
 *   Neumann and periodic need n_t with prime factors <= 13 (FPG_EUNSUPPORTED).
 * Each solve is the transform along t (two real lines per complex FFT), one
 * Thomas solve per mode along s, and the inverse transform; 1 <= n_s <= 4096.
 *
 * A plan holds the tables (built on the host in FP64 and copied once) and the
 * scratch for up to nvec rectangles in the caller's device workspace (>=
 * fpg_rect_plan_bytes; owned by the caller, valid until the plan is destroyed);
 * the plan handle is host memory.  fpg_rect_plan_create synchronises `stream`
 * once; fpg_rect_solve only enqueues on it (a cudaStream_t, NULL = default).
 * Errors: FPG_EINVAL (kind, sizes, h <= 0, kappa > 0, null pointers, nvec above
 * the plan's), FPG_ENOMEM (workspace short), FPG_EUNSUPPORTED, FPG_ECUDA. */
typedef enum { FPG_RECT_DIRICHLET = 0, FPG_RECT_NEUMANN = 1, FPG_RECT_PERIODIC = 2 } fpg_rect_kind;
typedef struct fpg_rect_plan fpg_rect_plan;
fpg_status fpg_rect_plan_bytes(int32_t kind, int32_t nt, int32_t ns, int32_t nvec, size_t* bytes);
fpg_status fpg_rect_plan_create(int32_t kind, int32_t nt, int32_t ns, double h, double kappa, int32_t nvec,
                                void* workspace, size_t bytes, void* stream, fpg_rect_plan** out);
fpg_status fpg_rect_solve(fpg_rect_plan* plan, const double* v, double* z, int32_t nvec);
void fpg_rect_plan_destroy(fpg_rect_plan* plan);

/* ---- 3-D box fast solve (the 3-D extension named after Sec. 2.1) -----------
 * z = A^{-1} v for nvec boxes of nx x ny x nz points (x fastest, then y, then z;
 * FP64, device pointers, v and z may not alias): the 7-point stencil with
 * spacing h in all directions (delta = 1/h^2), kappa <= 0 on the diagonal,
 * zero Dirichlet data one step beyond every face.  One more transform turns the
 * 3-D equation into independent 2-D ones: DST-I along x, DST-I along y (the a1
 * engines), one Thomas solve along z per mode pair (kx, ky) with diagonal
 * -6 delta + 2 delta cos(kx pi/(nx+1)) + 2 delta cos(ky pi/(ny+1)) + kappa, and the
 * two inverse transforms.  2 <= nx, ny <= 4096, 1 <= nz <= 4096, nvec * nx <= 65535.
 * Plan, workspace, stream and error rules as for the rectangle plans. */
typedef struct fpg_box_plan fpg_box_plan;
fpg_status fpg_box_plan_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t nvec, size_t* bytes);
fpg_status fpg_box_plan_create(int32_t nx, int32_t ny, int32_t nz, double h, double kappa, int32_t nvec,
                               void* workspace, size_t bytes, void* stream, fpg_box_plan** out);
fpg_status fpg_box_solve(fpg_box_plan* plan, const double* v, double* z, int32_t nvec);
void fpg_box_plan_destroy(fpg_box_plan* plan);

/* One-call forms (plan, solve, release; the tables are rebuilt at every call):
 * Neumann rectangles (Sec. 2.2, Eq. "submat_Neumann") and periodic rectangles
 * (Eq. "submat_Periodic") as described above; workspace >= the matching
 * *_workspace_bytes (= fpg_rect_plan_bytes of that kind).  Same errors. */
fpg_status fpg_neumann_workspace_bytes(int32_t nt, int32_t ns, int32_t nvec, size_t* bytes);
fpg_status fpg_neumann_solve(int32_t nt, int32_t ns, double h, double kappa, const double* v, double* z,
                             int32_t nvec, void* workspace, size_t bytes, void* stream);
fpg_status fpg_periodic_workspace_bytes(int32_t nt, int32_t ns, int32_t nvec, size_t* bytes);
fpg_status fpg_periodic_solve(int32_t nt, int32_t ns, double h, double kappa, const double* v, double* z,
                              int32_t nvec, void* workspace, size_t bytes, void* stream);

/* Element-wise conversion between FP64 and FP32 on the device, done with the
 * integer-pipe routines of the mixed-precision path (GB300 runs the hardware
 * conversion on its FP64 pipe).  (in_prec, out_prec) is (64, 32): round to
 * nearest even, magnitudes below 2^-126 give a signed zero, 2^128 and above,
 * inf and NaN give inf; or (32, 64): exact, binary32 subnormals give a signed
 * zero.  in and out are device arrays of count elements; the kernel runs on
 * `stream` (a cudaStream_t, NULL = default stream).  FPG_EINVAL on null
 * pointers, count < 0 or another precision pair. */
fpg_status fpg_convert(const void* in, int32_t in_prec, void* out, int32_t out_prec, int64_t count, void* stream);

/* Kernels the preconditioner of this domain runs for the centre block:
 * 0 = generic FFT engine (k_fft_forward, k_thomas_reg, k_fft_inverse),
 * 1 = size-specialised line DST (k_dst_lines_fwd, k_thomas_reg, k_dst_lines_inv;
 *     n = 64, 256, 512 in FP64 -- when the batch of nrhs centre blocks is large
 *     enough to fill the GPU -- and also 1024 in FP32),
 * 2 = dense DST (lengths with no FFT plan), 3 = fused one-pass cluster kernel
 * (FPG_OPT_FUSED_FASTSOLVE), 4 = no fast solve (identity or Jacobi). */
fpg_status fpg_fast_solve_path(fpg_domain* d, int32_t* path);

/* Launch shape of the Arnoldi step (a3 + a4) this domain's solve runs with its
 * current options: *kind 1 = register-resident cluster kernel
 * (k_arnoldi_cluster_reg, stencil fused), 2 = cluster kernel with w in HBM
 * (k_arnoldi_cluster), 0 = multi-launch MGS (no cluster); *cluster = CTAs per
 * right-hand side (0 for kind 0), *threads = threads per CTA, *ctas = CTAs of one
 * launch over all nrhs right-hand sides.  Any output pointer may be NULL.
 * FPG_EINVAL on a null handle. */
fpg_status fpg_arnoldi_shape(fpg_domain* d, int32_t* kind, int32_t* cluster, int32_t* threads, int32_t* ctas);

/* FMA throughput of this GPU measured by a short library kernel (FLOP/s,
 * 2 per FMA): precision 64 or 32.  Used as the ALU roofline. */
fpg_status fpg_probe_fma_peak(int32_t precision, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* FPG_H */
