"""Seeded synthetic inputs for the block-domain Helmholtz-Poisson solver.

This module is the one piece shared by the CPU oracle and the CUDA path: it
turns (geometry, n, kappa, seed) into right-hand-side vectors f in the library's
block-order layout. It contains none of the solver's arithmetic (no operator, no
transform, no Krylov step) -- only the definition of the synthetic workloads.

Layout (the library's I/O convention, the same one `include/fpg.h` documents):
  * One instance has one grid size n; the spacing is h = 1/(n+1).
  * Blocks are stored one after another: the centre C, then the arms present in
    the geometry in the order W, E, S, N.
      cross = C, W, E, S, N    T = C, W, E, S    L = C, E, N
  * C = [0,1]^2 holds the n x n nodes (i h, j h), i, j = 1..n.
  * Each arm owns the grid line it shares with C, so W and E hold (n+1) x n
    nodes (n+1 along x) and S and N hold n x (n+1) nodes (n+1 along y):
      W: x = -1 + i h, i = 1..n+1        E: x = 1 + (i-1) h, i = 1..n+1
      S: y = -1 + j h, j = 1..n+1        N: y = 1 + (j-1) h, j = 1..n+1
  * Inside a block the values are row-major with x fastest.

Workloads (synthetic; the paper uses no external data, Sec. 3):
  * "manufactured": p = sin(pi x) sin(pi y) exp(0.3 x), which vanishes on every
    edge of the L, T and cross domains (all edges lie on integer coordinates), so
    the Dirichlet data is zero and f = lap(p) + kappa p in closed form.
  * "fourier": per block, 16 modes sin(kx pi xi) sin(ky pi eta) / (kx^2 + ky^2)
    with N(0,1) coefficients and (kx, ky) uniform on {1..8}^2, in block-local
    coordinates (xi, eta) in [0,1]^2; generator numpy PCG64 seeded with
    seed*1000 + block_id.  Zero on every block edge.
"""
from __future__ import annotations

import math

import numpy as np

GEOMETRY_BLOCKS = {
    "cross": ("C", "W", "E", "S", "N"),
    "T": ("C", "W", "E", "S"),
    "L": ("C", "E", "N"),
}
GEOMETRY_CODE = {"L": 0, "T": 1, "cross": 2}
BLOCK_ID = {"C": 0, "W": 1, "E": 2, "S": 3, "N": 4}
# Box [x0, x1] x [y0, y1] of each block, in units of the centre block's side.
BLOCK_BOX = {
    "C": (0.0, 1.0, 0.0, 1.0),
    "W": (-1.0, 0.0, 0.0, 1.0),
    "E": (1.0, 2.0, 0.0, 1.0),
    "S": (0.0, 1.0, -1.0, 0.0),
    "N": (0.0, 1.0, 1.0, 2.0),
}


def block_shape(name: str, n: int) -> tuple[int, int]:
    """(nx, ny) of a block: C is n x n, W/E are (n+1) x n, S/N are n x (n+1)."""
    if name == "C":
        return n, n
    if name in ("W", "E"):
        return n + 1, n
    return n, n + 1


def block_first_node(name: str, n: int) -> tuple[int, int]:
    """Integer grid coordinates (I, J) of the block's node with i = j = 1;
    the physical position is (I h, J h) with h = 1/(n+1)."""
    m = n + 1
    return {
        "C": (1, 1),
        "W": (-m + 1, 1),
        "E": (m, 1),
        "S": (1, -m + 1),
        "N": (1, m),
    }[name]


def block_coords(name: str, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Physical x, y of every node of a block, shaped (ny, nx) (x fastest)."""
    nx, ny = block_shape(name, n)
    i0, j0 = block_first_node(name, n)
    h = 1.0 / (n + 1)
    xs = (i0 + np.arange(nx)) * h
    ys = (j0 + np.arange(ny)) * h
    return np.meshgrid(xs, ys, indexing="xy")


def total_unknowns(geometry: str, n: int) -> int:
    return sum(int(np.prod(block_shape(b, n))) for b in GEOMETRY_BLOCKS[geometry])


def manufactured_solution(geometry: str, n: int) -> np.ndarray:
    """p = sin(pi x) sin(pi y) exp(0.3 x) at every unknown, in block order."""
    parts = []
    for b in GEOMETRY_BLOCKS[geometry]:
        x, y = block_coords(b, n)
        parts.append((np.sin(math.pi * x) * np.sin(math.pi * y) * np.exp(0.3 * x)).ravel())
    return np.concatenate(parts)


def manufactured_rhs(geometry: str, n: int, kappa: float = 0.0) -> np.ndarray:
    """f = lap(p) + kappa p for the manufactured p, in block order."""
    parts = []
    pi = math.pi
    for b in GEOMETRY_BLOCKS[geometry]:
        x, y = block_coords(b, n)
        e = np.exp(0.3 * x)
        lap = e * np.sin(pi * y) * ((0.09 - 2.0 * pi * pi) * np.sin(pi * x) + 0.6 * pi * np.cos(pi * x))
        p = np.sin(pi * x) * np.sin(pi * y) * e
        parts.append((lap + kappa * p).ravel())
    return np.concatenate(parts)


def fourier_rhs(geometry: str, n: int, seed: int, modes: int = 16, kmax: int = 8) -> np.ndarray:
    """Random smooth right-hand side (see module docstring), in block order."""
    parts = []
    for b in GEOMETRY_BLOCKS[geometry]:
        rng = np.random.default_rng(seed * 1000 + BLOCK_ID[b])
        kx = rng.integers(1, kmax + 1, size=modes)
        ky = rng.integers(1, kmax + 1, size=modes)
        c = rng.standard_normal(modes)
        x, y = block_coords(b, n)
        x0, x1, y0, y1 = BLOCK_BOX[b]
        xi = (x - x0) / (x1 - x0)
        eta = (y - y0) / (y1 - y0)
        f = np.zeros_like(x)
        for q in range(modes):
            f += c[q] * np.sin(kx[q] * math.pi * xi) * np.sin(ky[q] * math.pi * eta) / (kx[q] ** 2 + ky[q] ** 2)
        parts.append(f.ravel())
    return np.concatenate(parts)


def rhs_batch(geometry: str, n: int, seeds, kind: str = "fourier", kappa: float = 0.0) -> np.ndarray:
    """Stack of right-hand sides, shape (len(seeds), total_unknowns)."""
    rows = []
    for s in seeds:
        if kind == "fourier":
            rows.append(fourier_rhs(geometry, n, int(s)))
        elif kind == "manufactured":
            rows.append(manufactured_rhs(geometry, n, kappa))
        else:
            raise ValueError(f"unknown workload kind {kind!r}")
    return np.ascontiguousarray(np.stack(rows))


def random_block_vectors(nvec: int, size: int, seed: int) -> np.ndarray:
    """Plain N(0,1) test vectors (operator-level parity inputs), shape (nvec, size)."""
    return np.random.default_rng(seed).standard_normal((nvec, size))


def serving_requests(count: int, rate_per_s: float, seed: int = 0,
                     sizes=(64, 128, 256, 512, 1024), max_rhs: int = 8):
    """Poisson-arrival request stream: list of dicts with arrival time (s),
    geometry, n, number of RHS, kappa and a per-request seed."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    geoms = ("L", "T", "cross")
    reqs = []
    for i in range(count):
        reqs.append({
            "id": i,
            "arrival_s": float(t[i]),
            "geometry": geoms[int(rng.integers(0, 3))],
            "n": int(sizes[int(rng.integers(0, len(sizes)))]),
            "nrhs": int(rng.integers(1, max_rhs + 1)),
            "kappa": (0.0, -10.0)[int(rng.integers(0, 2))],
            "seed": int(rng.integers(0, 2**31 - 1)),
        })
    return reqs


def fourier_rhs_torch(geometry: str, n: int, seed: int, device="cuda", modes: int = 16, kmax: int = 8):
    """fourier_rhs evaluated with torch on `device` (same coefficient draws, same
    formula; used where many large inputs are needed quickly, e.g. a request
    stream).  Returns a float64 tensor in block order."""
    import torch
    parts = []
    for b in GEOMETRY_BLOCKS[geometry]:
        rng = np.random.default_rng(seed * 1000 + BLOCK_ID[b])
        kx = rng.integers(1, kmax + 1, size=modes)
        ky = rng.integers(1, kmax + 1, size=modes)
        c = rng.standard_normal(modes)
        nx, ny = block_shape(b, n)
        i0, j0 = block_first_node(b, n)
        h = 1.0 / (n + 1)
        x0, x1, y0, y1 = BLOCK_BOX[b]
        xs = (i0 + torch.arange(nx, dtype=torch.float64, device=device)) * h
        ys = (j0 + torch.arange(ny, dtype=torch.float64, device=device)) * h
        xi = (xs - x0) / (x1 - x0)
        eta = (ys - y0) / (y1 - y0)
        sx = torch.sin(torch.as_tensor(kx, dtype=torch.float64, device=device)[:, None] * math.pi * xi[None, :])
        sy = torch.sin(torch.as_tensor(ky, dtype=torch.float64, device=device)[:, None] * math.pi * eta[None, :])
        w = torch.as_tensor(c / (kx ** 2 + ky ** 2), dtype=torch.float64, device=device)
        parts.append(torch.einsum("q,qy,qx->yx", w, sy, sx).reshape(-1))
    return torch.cat(parts)


# ---- the Neumann-sided cross (cell-centred grid) -------------------------------
# Boundary pattern of the paper's precision validation (Sec. 3.1): zero Dirichlet
# at the far ends of the four arms (x = -1, x = 2, y = -1, y = 2), zero normal
# derivative on the arms' sides.  Cell-centred grid, h = 1/n: every block holds
# n x n cell centres, block order C, W, E, S, N, x fastest; block b covers the
# unit square with lower-left corner NCROSS_CORNER[b].

NCROSS_CORNER = {"C": (0, 0), "W": (-1, 0), "E": (1, 0), "S": (0, -1), "N": (0, 1)}


def ncross_block_coords(name: str, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Cell centres x, y of one block of the Neumann-sided cross, shaped (n, n)."""
    x0, y0 = NCROSS_CORNER[name]
    c = (np.arange(n) + 0.5) / n
    return np.meshgrid(x0 + c, y0 + c)


def _ncross_psi(t):
    """The cubic through (-1, 0), (0, pi/2), (1, 3 pi/2), (2, 2 pi) and its first
    two derivatives (coefficients written out in powers of t)."""
    a0, a1, a2, a3 = math.pi / 2, 11 * math.pi / 12, math.pi / 4, -math.pi / 6
    return (a0 + t * (a1 + t * (a2 + t * a3)), a1 + t * (2 * a2 + 3 * a3 * t), 2 * a2 + 6 * a3 * t)


def ncross_validation_solution(n: int) -> np.ndarray:
    """p = sin(psi(x)) sin(psi(y)) at every cell centre, block order."""
    parts = []
    for b in ("C", "W", "E", "S", "N"):
        x, y = ncross_block_coords(b, n)
        parts.append((np.sin(_ncross_psi(x)[0]) * np.sin(_ncross_psi(y)[0])).ravel())
    return np.concatenate(parts)


def ncross_validation_rhs(n: int, kappa: float = 0.0) -> np.ndarray:
    """f = lap(p) + kappa p of the validation solution, block order."""
    parts = []
    for b in ("C", "W", "E", "S", "N"):
        x, y = ncross_block_coords(b, n)
        px, dx, ddx = _ncross_psi(x)
        py, dy, ddy = _ncross_psi(y)
        sx, sy = np.sin(px), np.sin(py)
        sxx = -sx * dx * dx + np.cos(px) * ddx
        syy = -sy * dy * dy + np.cos(py) * ddy
        parts.append((sxx * sy + sx * syy + kappa * sx * sy).ravel())
    return np.concatenate(parts)


def ncross_fourier_rhs(n: int, seed: int, modes: int = 16, kmax: int = 8) -> np.ndarray:
    """The "fourier" workload on the cell-centred blocks (same draws per block)."""
    parts = []
    for b in ("C", "W", "E", "S", "N"):
        rng = np.random.default_rng(seed * 1000 + BLOCK_ID[b])
        kx = rng.integers(1, kmax + 1, size=modes)
        ky = rng.integers(1, kmax + 1, size=modes)
        c = rng.standard_normal(modes)
        x, y = ncross_block_coords(b, n)
        x0, y0 = NCROSS_CORNER[b]
        xi, eta = x - x0, y - y0
        f = np.zeros_like(x)
        for q in range(modes):
            f += c[q] * np.sin(kx[q] * math.pi * xi) * np.sin(ky[q] * math.pi * eta) / (kx[q] ** 2 + ky[q] ** 2)
        parts.append(f.ravel())
    return np.concatenate(parts)


# ---- the chain of K crosses (several coupled blocks; vertex-centred, h = 1/(n+1)) ----
# 2K - 1 unit squares in a row along x (centres at even q, links at odd q), arms W
# and E at the ends and S_i, N_i below and above centre i (at q = 2(i-1)).  Block
# order: the coupled row as one rectangle ((2K-1)(n+1) - 1 columns, n rows), W, E
# ((n+1) x n), S_1..S_K, N_1..N_K (n x (n+1)); the arms own the line they share
# with the row.

def strip_block_boxes(K: int, n: int):
    """(name, first x node, first y node, nx, ny, unit-square corner) per block;
    node coordinates in units of h."""
    m = n + 1
    q = 2 * K - 1
    out = [("C", 1, 1, q * m - 1, n, None), ("W", -m + 1, 1, m, n, (-1, 0)), ("E", q * m, 1, m, n, (q, 0))]
    out += [(f"S{i}", 2 * (i - 1) * m + 1, -m + 1, n, m, (2 * (i - 1), -1)) for i in range(1, K + 1)]
    out += [(f"N{i}", 2 * (i - 1) * m + 1, m, n, m, (2 * (i - 1), 1)) for i in range(1, K + 1)]
    return out


def strip_total_unknowns(K: int, n: int) -> int:
    return ((2 * K - 1) * (n + 1) - 1) * n + (2 * K + 2) * n * (n + 1)


def strip_manufactured_rhs(K: int, n: int, kappa: float = 0.0) -> np.ndarray:
    """f = lap(p) + kappa p for p = sin(pi x) sin(pi y) exp(0.3 x) (zero on every
    integer line, so on the strip's edge), block order."""
    h = 1.0 / (n + 1)
    parts = []
    for _, i0, j0, nx, ny, _ in strip_block_boxes(K, n):
        x, y = np.meshgrid((i0 + np.arange(nx)) * h, (j0 + np.arange(ny)) * h)
        e = np.exp(0.3 * x)
        p = np.sin(math.pi * x) * np.sin(math.pi * y) * e
        lap = e * np.sin(math.pi * y) * ((0.09 - 2 * math.pi ** 2) * np.sin(math.pi * x)
                                          + 0.6 * math.pi * np.cos(math.pi * x))
        parts.append((lap + kappa * p).ravel())
    return np.concatenate(parts)


def strip_manufactured_solution(K: int, n: int) -> np.ndarray:
    h = 1.0 / (n + 1)
    parts = []
    for _, i0, j0, nx, ny, _ in strip_block_boxes(K, n):
        x, y = np.meshgrid((i0 + np.arange(nx)) * h, (j0 + np.arange(ny)) * h)
        parts.append((np.sin(math.pi * x) * np.sin(math.pi * y) * np.exp(0.3 * x)).ravel())
    return np.concatenate(parts)


def strip_fourier_rhs(K: int, n: int, seed: int, modes: int = 16, kmax: int = 8) -> np.ndarray:
    """The "fourier" workload per unit square of the chain (the coupled row takes
    square q's draws on its part x in [q, q+1]), block order."""
    h = 1.0 / (n + 1)
    parts = []
    for name, i0, j0, nx, ny, corner in strip_block_boxes(K, n):
        x, y = np.meshgrid((i0 + np.arange(nx)) * h, (j0 + np.arange(ny)) * h)
        f = np.zeros_like(x)
        if corner is None:
            sq = np.minimum(np.floor(x).astype(int), 2 * K - 2)  # square index of each column
            for i in range(2 * K - 1):
                f += np.where(sq == i, _square_modes(seed, 100 + i, x - i, y, modes, kmax), 0.0)
        else:
            block_id = _STRIP_ID[name[0]] * 16 + int(name[1:] or 0)
            f = _square_modes(seed, block_id, x - corner[0], y - corner[1], modes, kmax)
        parts.append(f.ravel())
    return np.concatenate(parts)


_STRIP_ID = {"W": 1, "E": 2, "S": 3, "N": 4}


def _square_modes(seed, block_id, xi, eta, modes, kmax):
    rng = np.random.default_rng(seed * 1000 + block_id)
    kx = rng.integers(1, kmax + 1, size=modes)
    ky = rng.integers(1, kmax + 1, size=modes)
    c = rng.standard_normal(modes)
    f = np.zeros_like(xi)
    for q in range(modes):
        f += c[q] * np.sin(kx[q] * math.pi * xi) * np.sin(ky[q] * math.pi * eta) / (kx[q] ** 2 + ky[q] ** 2)
    return f


# --------------------------------------------------------------------- lattices
# A general concatenated geometry: any edge-connected set of unit squares
# [i, i+1] x [j, j+1], 0 <= i, j < 8, given as a 64-bit mask (bit i + 8 j).
# Block order (the library's I/O convention for FPG_GEOM_LATTICE): coupled
# squares (two or more edge neighbours; of a lone pair, the first) in bit order,
# n x n each; the links (grid lines shared by two coupled squares: vertical
# edges by (j, i) of the left square, then horizontal edges by (j, i) of the
# lower square), n points each; the junction points (lattice vertices with all
# four squares around them, by (Y, X)); then the independent squares (one
# neighbour) in bit order, each with the line it shares with its neighbour,
# last (neighbour east or north) or first (west or south): (n+1) x n or n x (n+1).

LATTICE_EXAMPLES = {
    "square2x2": (1 << 0) | (1 << 1) | (1 << 8) | (1 << 9),
    "L5": (1 << 0) | (1 << 1) | (1 << 2) | (1 << 8) | (1 << 16),          # L-shaped coupled set
    "T6": (1 << 0) | (1 << 1) | (1 << 2) | (1 << 3) | (1 << 4) | (1 << 10),  # a row with a stem
    "cross": (1 << 9) | (1 << 8) | (1 << 10) | (1 << 1) | (1 << 17),
    "domino": (1 << 0) | (1 << 1),
}


def lattice_squares(mask: int):
    return [(b % 8, b // 8) for b in range(64) if (mask >> b) & 1]


def lattice_blocks(mask: int, n: int):
    """(kind, (i, j) or None, first x node, first y node, nx, ny) per block in block
    order; kind is 'Q' (coupled square), 'V'/'H' (link), 'P' (junction) or 'A'
    (independent square); node coordinates in units of h."""
    m = n + 1
    have = set(lattice_squares(mask))
    nb = {s: [d for d in ((1, 0), (-1, 0), (0, 1), (0, -1)) if (s[0] + d[0], s[1] + d[1]) in have]
          for s in have}
    order = lattice_squares(mask)
    coupled = [s for s in order if len(nb[s]) >= 2] or order[:1]
    cset = set(coupled)
    out = [("Q", s, s[0] * m + 1, s[1] * m + 1, n, n) for s in coupled]
    for kind, d in (("V", (1, 0)), ("H", (0, 1))):
        for j in range(8):
            for i in range(8):
                if (i, j) in cset and (i + d[0], j + d[1]) in cset:
                    if kind == "V":
                        out.append(("V", (i, j), (i + 1) * m, j * m + 1, 1, n))
                    else:
                        out.append(("H", (i, j), i * m + 1, (j + 1) * m, n, 1))
    for Y in range(1, 8):
        for X in range(1, 8):
            if {(X - 1, Y - 1), (X, Y - 1), (X - 1, Y), (X, Y)} <= have:
                out.append(("P", (X, Y), X * m, Y * m, 1, 1))
    for s in order:
        if s in cset:
            continue
        d = nb[s][0]
        i, j = s
        box = {(1, 0): (i * m + 1, j * m + 1, m, n), (-1, 0): (i * m, j * m + 1, m, n),
               (0, 1): (i * m + 1, j * m + 1, n, m), (0, -1): (i * m + 1, j * m, n, m)}[d]
        out.append(("A", s) + box)
    return out


def lattice_total_unknowns(mask: int, n: int) -> int:
    return sum(b[4] * b[5] for b in lattice_blocks(mask, n))


def _lattice_xy(mask: int, n: int):
    h = 1.0 / (n + 1)
    xs, ys = [], []
    for _, _, i0, j0, nx, ny in lattice_blocks(mask, n):
        x, y = np.meshgrid((i0 + np.arange(nx)) * h, (j0 + np.arange(ny)) * h)
        xs.append(x.ravel())
        ys.append(y.ravel())
    return np.concatenate(xs), np.concatenate(ys)


def lattice_manufactured_solution(mask: int, n: int) -> np.ndarray:
    """p = sin(pi x) sin(pi y) exp(0.3 x) at every unknown (zero on every integer
    line, so on the union's edge), block order."""
    x, y = _lattice_xy(mask, n)
    return np.sin(math.pi * x) * np.sin(math.pi * y) * np.exp(0.3 * x)


def lattice_manufactured_rhs(mask: int, n: int, kappa: float = 0.0) -> np.ndarray:
    x, y = _lattice_xy(mask, n)
    e = np.exp(0.3 * x)
    lap = e * np.sin(math.pi * y) * ((0.09 - 2 * math.pi ** 2) * np.sin(math.pi * x)
                                      + 0.6 * math.pi * np.cos(math.pi * x))
    return lap + kappa * np.sin(math.pi * x) * np.sin(math.pi * y) * e


def lattice_fourier_rhs(mask: int, n: int, seed: int, modes: int = 16, kmax: int = 8) -> np.ndarray:
    """The "fourier" workload per unit square (seeded by seed * 1000 + 100 + bit),
    in block order; every point on a grid line between squares gets 0 (each
    square's modes vanish on its edges)."""
    m = n + 1
    h = 1.0 / m
    parts = []
    for _, _, i0, j0, nx, ny in lattice_blocks(mask, n):
        I, J = np.meshgrid(i0 + np.arange(nx), j0 + np.arange(ny))
        f = np.zeros(I.shape)
        inside = (I % m != 0) & (J % m != 0)
        for (si, sj) in set(zip((I[inside] // m).tolist(), (J[inside] // m).tolist())):
            sel = inside & (I // m == si) & (J // m == sj)
            f[sel] = _square_modes(seed, 100 + si + 8 * sj, I[sel] * h - si, J[sel] * h - sj, modes, kmax)
        parts.append(f.ravel())
    return np.concatenate(parts)
