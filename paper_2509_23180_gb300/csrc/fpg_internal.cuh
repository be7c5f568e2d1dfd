// Internal declarations shared by the library's translation units.
// Nothing here crosses the C ABI (include/fpg.h is the public surface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fpg.h"
#include "fpg_dst.cuh"
#include "fpg_once.h"

namespace fpg {

// ---------------------------------------------------------------------------
// Batch of blocks of one shape inside larger vectors.  Block b of a launch lives
// at base + (b / nper) * rhs_stride + off[b % nper]: nper <= 8 blocks per
// right-hand side (e.g. the two arms W and E), one right-hand side after another.
struct BatchDesc {
  long long rhs_stride;
  long long off[8];
  int nper;
};

// Memory layout of one block kind, seen as "lines": the fast solve transforms
// along t (length nt) and runs the tridiagonal sweep along s (length ns).
// Element (t, s) sits at t * st + s * ss inside the block.
struct LineLayout {
  int nt, ns;
  long long st, ss;
};

// Rows per lane of the register Thomas kernel for a sweep of ns rows: the smallest
// compiled chunk covering ns / 32 (0: the sweep is too long for it).
__host__ __device__ inline int thomas_chunk_rows(int ns) {
  const int need = (ns + 31) / 32;
  const int chunks[] = {1, 2, 3, 4, 5, 8, 9, 12, 16, 17, 24, 32, 33};
  for (int c : chunks)
    if (need <= c) return c;
  return 0;
}

// Everything the fast-solve kernels need for one block kind.
struct FastSolveTables {
  int n;              // transform length (= domain n)
  int ns;             // sweep length
  double delta;       // 1/h^2
  DstPlan plan;       // DST-I plan and tables in the compute precision
  const void* rpiv;   // Thomas reciprocal pivots r_s, [n][ns] (s fastest), compute precision
  const void* mneg;   // -delta r_s, [n][ns], compute precision
  // FP64 only (else null): running products of mneg inside each lane's chunk of
  // thomas_chunk_rows(ns) rows, from the chunk's first row (pfwd) and from its last
  // (pbwd), [n][ns]: the products the Thomas kernel's carry fix-ups would form
  const void* pfwd = nullptr;
  const void* pbwd = nullptr;
  int use_products = 1;  // 0: the kernel forms those products itself (same bits)
  int q = 0;          // line pairs per CTA in the DST kernels (0: built-in choice)
  int mt = 0;         // warps (= modes) per CTA in the Thomas kernel (0: 8)
  int fused = 0;      // 1: one-pass cluster kernel when the block fits
  int generic = 0;    // DST engine: 0 auto, 1 generic FFT engine, 2 size-specialised where compiled
  int bulk = 0;       // 1: FP32 forward DST as the persistent kernel with bulk asynchronous row copies
  int cluster = 0;             // 1: FP32 one-pass cluster kernel where it fits (fpg_cluster_fs.cu)
  const void* cl_sigma = nullptr;  // its tables (FP32): sigma_k and the scaled pivot at each strip start
  const void* cl_wseed = nullptr;
  int* err = nullptr;          // device status word: a bounded wait that gave up writes 1 (null: none)
  int wait_limit = 1 << 22;    // tries of every bounded device wait (0: give up at once)
  int kind = 0;       // transform along t: 0 DST-I (Dirichlet ends), 1 DCT-II (Neumann ends), 2 real DFT
                      // (periodic); 1 and 2 FP64 only
  const void* post = nullptr;  // DCT-II: e^{-i pi k/(2n)}, k < n (complex, FP64)
};

// Offsets of the arm blocks W, E, S, N inside one full vector (-1 = absent),
// and the arm shape: every arm is n lines across (along its interface) by `as`
// lines along its sweep (n + 1 on the vertex-centred grid, whose arms own the
// line they share with the centre; n on the cell-centred grid).  bc = 0: every
// edge Dirichlet (zero neighbour); bc = 1: cell-centred, the arms' sides are
// Neumann faces (ghost = the cell's value) and their far ends Dirichlet faces
// (ghost = minus the cell's value).
struct ArmOffsets {
  long long off[4];
  int as = 0;
  int bc = 0;
};

// The chain of K crosses (2 <= K <= 5): the coupled row is nxc = (2K-1)(n+1) - 1
// columns by n rows; its arms, in slot order W, E, S_1..S_K, N_1..N_K, start at
// off[slot] inside one full vector (W and E (n+1) x n, S and N n x (n+1)).
struct ChainGeom {
  int K = 0, n = 0, nxc = 0;
  long long off[12];
};

// Tables for the interface (Schur) correction, reduced form:
// G_a = delta^2 Q diag(g_k) Q^T = Toeplitz-plus-Hankel with entries
// T(|i-j|) - H(i+j) (0-based i, j), stored as T[0..2n+1] followed by H[0..2n-1]:
// DST-I arms H(m) = T(m+2); DCT-II arms H(m) = -T(m+1).
// A general concatenated geometry (FPG_GEOM_LATTICE, fpg_lattice.cu): counts and
// block offsets.  The coupled set -- coupled squares (n x n each, offsets sq_off),
// links (n points each, from link_base) and junctions (one point each, from
// junc_base) -- is the prefix [0, nc) of a full vector; the independent squares
// follow, those whose neighbour is west or east ((n+1) x n, we_off) and those
// whose neighbour is south or north (n x (n+1), sn_off).
struct LatticeGeom {
  int n = 0, ncsq = 0, nlinks = 0, njunc = 0, nfaces = 0, nwe = 0, nsn = 0;
  long long nc = 0, ntot = 0, link_base = 0, junc_base = 0;
  long long sq_off[64] = {0};
  long long we_off[8] = {0}, sn_off[8] = {0};
};
// lattice_shape() and lattice_tables() (fpg_lattice_host.h) fill it; false: the
// mask is not an edge-connected set of at least two squares.

// Host tables of a lattice.  Coupled set (length nc): nbr = coupled indices of the
// W, E, S, N neighbours (-1: not in the coupled set); cf = up to two interface
// corrections (index face * n + position, -1: none); anb = global indices of up
// to two neighbouring points of independent squares.  Full vector (length ntot):
// gnbr = global indices of the four neighbours (-1: outside, zero Dirichlet);
// gcn = for a point of an independent square, its neighbour in the coupled set
// (-1: none).  faces = (offset of the coupled square, side 0 W / 1 E / 2 S / 3 N)
// facing each independent square; lpiv = reciprocal Thomas pivots of a link's
// own operator tridiag(delta, -4 delta + kappa, delta).
struct LatticeHost {
  std::vector<int4> nbr, gnbr;
  std::vector<int2> cf, anb, faces;
  std::vector<int> gcn;
  std::vector<double> lpiv;
};

// The same tables in the device workspace.
struct LatticeDev {
  long long nc = 0, link_base = 0, junc_base = 0;
  int nfaces = 0, nlinks = 0, njunc = 0;
  const int4* nbr = nullptr;
  const int2* cf = nullptr;
  const int2* anb = nullptr;
  const int2* faces = nullptr;
  const int4* gnbr = nullptr;
  const int* gcn = nullptr;
  const double* lpiv = nullptr;
};
cudaError_t launch_lattice_schur(const void* z, int zprec, long long zstride, double* w, long long wstride,
                                 const LatticeDev& t, int n, double delta, double kappa, const double* ctab,
                                 double* corr, const int* active, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_lattice_skeleton(const double* v, void* z, int zprec, const LatticeDev& t, int n, double delta,
                                    double kappa, const int* active, int nrhs, cudaStream_t st);
cudaError_t launch_lattice_reduce_rhs(const double* f, const double* q, long long ntot, const LatticeDev& t,
                                      double delta, double* fc, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_lattice_arm_rhs(const double* f, const double* u, long long ntot, const LatticeDev& t,
                                   double delta, double* out, double* p, int nrhs, int gx, cudaStream_t st);
cudaError_t launch_lattice_global_apply(const double* p, double* y, const double* f, long long ntot,
                                        const LatticeDev& t, double delta, double kappa, double* part, int gmax,
                                        int nrhs, int gx, double* rel_out, double* fnorm_out, double rtol,
                                        double* tolabs, cudaStream_t st);

struct SchurTables {
  const double* ctab;
};

// Device-side state of one domain's GMRES (all pointers into the workspace).
struct KrylovState {
  int nrhs, m, n;
  long long nc;           // n*n
  double* V;              // [m+1][nrhs][nc]
  void* Z;                // [m][nrhs][nc] (double or float)
  double* w;              // [nrhs][nc]
  double* u;              // [nrhs][nc] current centre iterate
  double* fc;             // [nrhs][nc] reduced right-hand side f'_c
  double* H;              // [nrhs][m][m+1] column-major Hessenberg
  double* cs;             // [nrhs][m]
  double* sn;             // [nrhs][m]
  double* g;              // [nrhs][m+1]
  double* y;              // [nrhs][m]
  double* part;           // [2][nrhs][gmax] reduction partials
  double* tolabs;         // [nrhs] rtol * ||f||
  double* fnorm;          // [nrhs] ||f||
  double* res;            // [nrhs] last |g_{j+1}|
  double* rnorm;          // [nrhs] last true Schur residual norm
  int* active;            // [nrhs] 1 while this right-hand side iterates in the cycle
  int* done;              // [nrhs] 1 once converged
  int* kcyc;              // [nrhs] Arnoldi steps taken in the current cycle
  int* iters;             // [nrhs] total steps
  int gx;                 // CTAs per right-hand side in point-wise kernels
};

// Error recording (thread-local text of the last CUDA error).
void record_cuda_error(cudaError_t e, const char* where);

}  // namespace fpg

#define FPG_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) {                                 \
      fpg::record_cuda_error(_e, #expr);                     \
      return FPG_ECUDA;                                      \
    }                                                        \
  } while (0)

#define FPG_TRY(x)               \
  do {                           \
    fpg_status _s = (x);         \
    if (_s != FPG_OK) return _s; \
  } while (0)

// ---------------------------------------------------------------------------
// Device helpers.
#ifdef __CUDACC__
namespace fpg {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  // Butterfly: every lane ends with the same total, the order is fixed.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of one double per thread (blockDim.x a multiple of
// 32, <= 1024).  Returns the total to every thread.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (lane < nw) ? red[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

// 5-point stencil sum (p_l + p_r + p_d + p_u - 4 p_c) written as the sum of the
// four differences (p_nb - p_c): for a smooth field each difference is exact
// (the operands are within a factor 2), so the rounding error is of the size of
// the differences instead of |p_c|; that keeps the residual f - K p meaningful
// down to ~1e-13 relative at h = 1/1025, where the plain sum loses ~5e-11.
// Neighbours on a Dirichlet edge are passed as 0.
__device__ __forceinline__ double stencil_sum(double c, double l, double r, double d, double u) {
  return ((l - c) + (r - c)) + ((d - c) + (u - c));
}

// Sum of cnt partials p[0..cnt) in a fixed order, done by one warp; every lane
// of the calling warp gets the total.
__device__ __forceinline__ double warp_sum_partials(const double* p, int cnt) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < cnt; i += 32) s += p[i];
  return warp_sum(s);
}

}  // namespace fpg
#endif
