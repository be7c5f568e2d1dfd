// Host layout of the general concatenated geometry (FPG_GEOM_LATTICE): which
// square is coupled or independent, every block's offset, a locator from grid
// point to unknown, and the neighbour / coupling tables the lattice kernels
// read (see fpg_lattice.cu for the partition and the block order).  Host code
// only; no heap in the layout itself (the tables are std::vectors).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fpg_internal.cuh"

namespace fpg {
namespace lattice_detail {

constexpr int kDir[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};  // W, E, S, N

inline bool present(uint64_t mask, int i, int j) {
  return i >= 0 && j >= 0 && i < 8 && j < 8 && ((mask >> (i + 8 * j)) & 1ULL);
}

inline int neighbour_count(uint64_t mask, int i, int j) {
  int c = 0;
  for (const auto& d : kDir) c += present(mask, i + d[0], j + d[1]) ? 1 : 0;
  return c;
}

// The whole layout of a lattice: which square is which, every block's offset,
// and a locator from grid point (I, J) to its global index (-1: not an unknown).
struct LatticeMap {
  uint64_t mask = 0;
  int n = 0, m = 0;
  int role[64];          // per bit: 0 absent, 1 coupled, 2 independent
  int dir[64];           // independent: direction to its neighbour (0 W, 1 E, 2 S, 3 N)
  long long off[64];     // block offset of every square
  long long vlink[64];   // offset of the link across the vertical edge right of square b (-1: none)
  long long hlink[64];   // offset of the link across the horizontal edge above square b (-1: none)
  long long junc[64];    // offset of the junction at vertex (X, Y), bit X + 8 Y (-1: none)
  int ncsq = 0, nlinks = 0, njunc = 0, nind = 0;
  long long nc = 0, ntot = 0;

  bool build(uint64_t msk, int nn) {
    mask = msk;
    n = nn;
    m = nn + 1;
    const long long nsq = (long long)n * n;
    int first = -1, count = 0;
    for (int b = 0; b < 64; ++b) {
      role[b] = 0;
      dir[b] = -1;
      off[b] = vlink[b] = hlink[b] = junc[b] = -1;
      if ((mask >> b) & 1ULL) {
        ++count;
        if (first < 0) first = b;
      }
    }
    if (count < 2) return false;
    // connected (edge adjacency)
    {
      uint64_t seen = 1ULL << first;
      bool grew = true;
      while (grew) {
        grew = false;
        for (int b = 0; b < 64; ++b) {
          if (!((seen >> b) & 1ULL)) continue;
          for (const auto& d : kDir) {
            const int i = b % 8 + d[0], j = b / 8 + d[1];
            if (present(mask, i, j) && !((seen >> (i + 8 * j)) & 1ULL)) {
              seen |= 1ULL << (i + 8 * j);
              grew = true;
            }
          }
        }
      }
      if (seen != mask) return false;
    }
    for (int b = 0; b < 64; ++b)
      if ((mask >> b) & 1ULL) role[b] = neighbour_count(mask, b % 8, b / 8) >= 2 ? 1 : 2;
    bool any = false;
    for (int b = 0; b < 64; ++b) any = any || role[b] == 1;
    if (!any) role[first] = 1;
    long long o = 0;
    for (int b = 0; b < 64; ++b)
      if (role[b] == 1) { off[b] = o; o += nsq; ++ncsq; }
    for (int j = 0; j < 8; ++j)
      for (int i = 0; i < 8; ++i) {
        const int b = i + 8 * j;
        if (role[b] == 1 && i + 1 < 8 && role[b + 1] == 1) { vlink[b] = o; o += n; ++nlinks; }
      }
    for (int j = 0; j < 8; ++j)
      for (int i = 0; i < 8; ++i) {
        const int b = i + 8 * j;
        if (role[b] == 1 && j + 1 < 8 && role[b + 8] == 1) { hlink[b] = o; o += n; ++nlinks; }
      }
    for (int Y = 1; Y < 8; ++Y)
      for (int X = 1; X < 8; ++X)
        if (present(mask, X - 1, Y - 1) && present(mask, X, Y - 1) && present(mask, X - 1, Y) && present(mask, X, Y)) {
          junc[X + 8 * Y] = o++;
          ++njunc;
        }
    nc = o;
    for (int b = 0; b < 64; ++b) {
      if (role[b] != 2) continue;
      for (int d = 0; d < 4; ++d)
        if (present(mask, b % 8 + kDir[d][0], b / 8 + kDir[d][1])) dir[b] = d;
      off[b] = o;
      o += (long long)n * m;
      ++nind;
    }
    ntot = o;
    return true;
  }

  // Global index of grid point (I, J) (units of h), -1 if it is not an unknown.
  long long locate(long long I, long long J) const {
    if (I < 0 || J < 0 || I >= 8LL * m || J >= 8LL * m) return -1;
    const int i = (int)(I / m), j = (int)(J / m), ri = (int)(I % m), rj = (int)(J % m);
    if (ri != 0 && rj != 0) {  // inside square (i, j)
      const int b = i + 8 * j;
      if (role[b] == 0) return -1;
      if (role[b] == 1) return off[b] + (long long)(rj - 1) * n + (ri - 1);
      switch (dir[b]) {
        case 1: return off[b] + (long long)(rj - 1) * m + (ri - 1);  // line last column (neighbour east)
        case 0: return off[b] + (long long)(rj - 1) * m + ri;        // line first column (west)
        case 3: return off[b] + (long long)(rj - 1) * n + (ri - 1);  // line last row (north)
        default: return off[b] + (long long)rj * n + (ri - 1);       // line first row (south)
      }
    }
    if (ri == 0 && rj != 0) {  // on the vertical line x = i, inside row j
      const int L = i - 1, R = i;
      if (!present(mask, L, j) || !present(mask, R, j)) return -1;
      const int bl = L + 8 * j, br = R + 8 * j;
      if (role[bl] == 1 && role[br] == 1) return vlink[bl] + (rj - 1);
      if (role[bl] == 2) return off[bl] + (long long)(rj - 1) * m + n;  // left square owns it (last column)
      return off[br] + (long long)(rj - 1) * m;                          // right square owns it (first column)
    }
    if (rj == 0 && ri != 0) {  // on the horizontal line y = j, inside column i
      const int D = j - 1, U = j;
      if (!present(mask, i, D) || !present(mask, i, U)) return -1;
      const int bd = i + 8 * D, bu = i + 8 * U;
      if (role[bd] == 1 && role[bu] == 1) return hlink[bd] + (ri - 1);
      if (role[bd] == 2) return off[bd] + (long long)n * n + (ri - 1);  // lower square owns it (last row)
      return off[bu] + (ri - 1);                                         // upper square owns it (first row)
    }
    if (i < 1 || j < 1) return -1;  // a lattice vertex
    return junc[i + 8 * j];
  }
};

}  // namespace lattice_detail

inline bool lattice_shape(uint64_t mask, int n, LatticeGeom* g) {
  lattice_detail::LatticeMap M;
  if (!M.build(mask, n)) return false;
  *g = LatticeGeom{};
  g->n = n;
  g->ncsq = M.ncsq;
  g->nlinks = M.nlinks;
  g->njunc = M.njunc;
  g->nfaces = M.nind;
  g->nc = M.nc;
  g->ntot = M.ntot;
  g->link_base = (long long)M.ncsq * n * n;
  g->junc_base = g->link_base + (long long)M.nlinks * n;
  int k = 0;
  for (int b = 0; b < 64; ++b) {
    if (M.role[b] == 1) {
      g->sq_off[k++] = M.off[b];
    } else if (M.role[b] == 2) {
      const bool we = M.dir[b] <= 1;
      if (we) {
        if (g->nwe < 8) g->we_off[g->nwe] = M.off[b];
        g->nwe++;
      } else {
        if (g->nsn < 8) g->sn_off[g->nsn] = M.off[b];
        g->nsn++;
      }
    }
  }
  return true;
}

// Host tables of a lattice (see fpg_internal.cuh for their meaning).
inline bool lattice_tables(uint64_t mask, int n, double delta, double kappa, LatticeHost* t) {
  lattice_detail::LatticeMap M;
  if (!M.build(mask, n)) return false;
  const long long nc = M.nc, ntot = M.ntot;
  t->nbr.assign((size_t)nc, make_int4(-1, -1, -1, -1));
  t->cf.assign((size_t)nc, make_int2(-1, -1));
  t->anb.assign((size_t)nc, make_int2(-1, -1));
  t->gnbr.assign((size_t)ntot, make_int4(-1, -1, -1, -1));
  t->gcn.assign((size_t)ntot, -1);
  t->faces.clear();
  // every unknown: its grid point, then its four neighbours
  auto visit = [&](long long I0, long long J0, int nx, int ny, long long base) {
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long long I = I0 + x, J = J0 + y, g = base + (long long)y * nx + x;
        const long long w = M.locate(I - 1, J), e = M.locate(I + 1, J), s = M.locate(I, J - 1), nn = M.locate(I, J + 1);
        t->gnbr[(size_t)g] = make_int4((int)w, (int)e, (int)s, (int)nn);
        if (g < nc) {
          auto cpl = [&](long long q) { return q >= 0 && q < nc ? (int)q : -1; };
          t->nbr[(size_t)g] = make_int4(cpl(w), cpl(e), cpl(s), cpl(nn));
          int2 a = make_int2(-1, -1);
          for (long long q : {w, e, s, nn})
            if (q >= nc) (a.x < 0 ? a.x : a.y) = (int)q;
          t->anb[(size_t)g] = a;
        } else {
          for (long long q : {w, e, s, nn})
            if (q >= 0 && q < nc) t->gcn[(size_t)g] = (int)q;
        }
      }
  };
  const long long m = M.m;
  for (int b = 0; b < 64; ++b) {
    const long long i = b % 8, j = b / 8;
    if (M.role[b] == 1) visit(i * m + 1, j * m + 1, n, n, M.off[b]);
  }
  for (int b = 0; b < 64; ++b)
    if (M.vlink[b] >= 0) visit((b % 8 + 1) * m, (b / 8) * m + 1, 1, n, M.vlink[b]);
  for (int b = 0; b < 64; ++b)
    if (M.hlink[b] >= 0) visit((b % 8) * m + 1, (b / 8 + 1) * m, n, 1, M.hlink[b]);
  for (int b = 0; b < 64; ++b)
    if (M.junc[b] >= 0) visit((b % 8) * m, (b / 8) * m, 1, 1, M.junc[b]);
  for (int b = 0; b < 64; ++b) {
    if (M.role[b] != 2) continue;
    const long long i = b % 8, j = b / 8;
    switch (M.dir[b]) {
      case 1: visit(i * m + 1, j * m + 1, (int)m, n, M.off[b]); break;
      case 0: visit(i * m, j * m + 1, (int)m, n, M.off[b]); break;
      case 3: visit(i * m + 1, j * m + 1, n, (int)m, M.off[b]); break;
      default: visit(i * m + 1, j * m, n, (int)m, M.off[b]); break;
    }
  }
  // faces: the coupled square next to each independent square, and the side of
  // it that faces the independent square (0 W, 1 E, 2 S, 3 N)
  for (int b = 0; b < 64; ++b) {
    if (M.role[b] != 2) continue;
    const int d = M.dir[b];
    const int cb = (b % 8 + lattice_detail::kDir[d][0]) + 8 * (b / 8 + lattice_detail::kDir[d][1]);
    const int side = d ^ 1;  // the neighbour's side facing back
    const int f = (int)t->faces.size();
    t->faces.push_back(make_int2((int)M.off[cb], side));
    for (int q = 0; q < n; ++q) {
      long long idx;
      switch (side) {
        case 0: idx = M.off[cb] + (long long)q * n; break;
        case 1: idx = M.off[cb] + (long long)q * n + n - 1; break;
        case 2: idx = M.off[cb] + q; break;
        default: idx = M.off[cb] + (long long)(n - 1) * n + q; break;
      }
      int2& c = t->cf[(size_t)idx];
      (c.x < 0 ? c.x : c.y) = f * n + q;
    }
  }
  // the links' own operator tridiag(delta, -4 delta + kappa, delta): reciprocal pivots
  t->lpiv.assign((size_t)n, 0.0);
  const double d0 = -4.0 * delta + kappa;
  double rp = 1.0 / d0;
  t->lpiv[0] = rp;
  for (int s = 1; s < n; ++s) {
    rp = 1.0 / (d0 - delta * delta * rp);
    t->lpiv[(size_t)s] = rp;
  }
  return true;
}

}  // namespace fpg
