"""Element-wise comparison for the GPU parity tests (test infrastructure).

`rel(a, b)` is the error measure of every parity assertion.  It is the largest of
  * the 2-norm relative error ||a - b||_2 / ||b||_2 over the whole array, and
  * for every vector (the last axis holds one vector; a 2-D array is a batch)
    the max-abs relative error max_i |a_i - b_i| / max_i |b_i|.
The second term is what makes the comparison element-wise: one wrong grid line
of a 328,704-point solution shows at its own size instead of being diluted by
the norm of the whole vector.

`part_errors(P, R, geometry, n)` splits a whole-domain vector in the library's
block order (centre C, then the arms W, E, S, N present) into its blocks and
its interface lines -- the arm's line next to C ("W|C") and C's edge line next
to the arm ("C|W") -- and gives max|a - b| / max|b| on each part (with b's
scale floored at 1% of the whole vector's), the maximum over the batch.  `assert_solution` checks `rel` and every part against one bar.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def _rows(a):
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(1, -1) if a.ndim <= 1 else a.reshape(-1, a.shape[-1])


def maxabs_rel(a, b) -> float:
    """max over vectors of max|a - b| / max|b| (a zero vector b asks for a == 0)."""
    A, Bv = _rows(a), _rows(b)
    assert A.shape == Bv.shape, (A.shape, Bv.shape)
    worst = 0.0
    for x, y in zip(A, Bv):
        scale = float(np.abs(y).max()) if y.size else 0.0
        diff = float(np.abs(x - y).max()) if y.size else 0.0
        worst = max(worst, diff / scale if scale > 0.0 else diff)
    return worst


def norm_rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / nb if nb > 0.0 else float(np.linalg.norm(a))


def rel(a, b) -> float:
    """The larger of the 2-norm relative error and the per-vector max-abs one."""
    return max(norm_rel(a, b), maxabs_rel(a, b))


def part_slices(geometry: str, n: int) -> list[tuple[str, np.ndarray]]:
    """(label, flat indices) of every block and interface line of a cross, T or L
    in block order.  Arms W and E are (n+1) x n with the interface column last
    (W) or first (E); S and N are n x (n+1) with the interface row last (S) or
    first (N); C is n x n."""
    parts = []
    off = 0
    offs = {}
    for name in W.GEOMETRY_BLOCKS[geometry]:
        nx, ny = W.block_shape(name, n)
        offs[name] = off
        parts.append((name, np.arange(off, off + nx * ny)))
        off += nx * ny
    j = np.arange(n)
    c_edge = {"W": j * n, "E": j * n + n - 1, "S": j, "N": (n - 1) * n + j}
    for name in W.GEOMETRY_BLOCKS[geometry][1:]:
        o = offs[name]
        arm_line = {"W": o + j * (n + 1) + n, "E": o + j * (n + 1),
                    "S": o + n * n + j, "N": o + j}[name]
        parts.append((f"{name}|C", arm_line))
        parts.append((f"C|{name}", c_edge[name]))
    return parts


PART_FLOOR = 0.01


def part_errors(P, R, geometry: str, n: int) -> dict[str, float]:
    """max|P - R| / scale on every part, the maximum over the batch.  The scale is
    the part's own max|R|, but at least PART_FLOOR (1%) of the whole vector's: a
    part whose values all lie far below the solution's size -- the interface
    lines of the manufactured solution sin(pi x) sin(pi y) e^{0.3x}, which
    vanishes on x, y in {0, 1} where those lines sit -- is judged at 1% of the
    solution's scale instead of at the size of its own near-zero values."""
    A, Bv = _rows(P), _rows(R)
    out = {}
    for label, idx in part_slices(geometry, n):
        worst = 0.0
        for x, y in zip(A, Bv):
            whole = float(np.abs(y).max()) if y.size else 0.0
            scale = max(float(np.abs(y[idx]).max()), PART_FLOOR * whole)
            diff = float(np.abs(x[idx] - y[idx]).max())
            worst = max(worst, diff / scale if scale > 0.0 else diff)
        out[label] = worst
    return out


def assert_solution(P, R, geometry: str, n: int, tol: float, what: str = "") -> dict[str, float]:
    """rel(P, R) <= tol and max|P - R| / max|R| <= tol on every block and interface line."""
    e = rel(P, R)
    parts = part_errors(P, R, geometry, n)
    bad = {k: v for k, v in parts.items() if not v <= tol}
    assert e <= tol and not bad, (what, geometry, n, e, bad or parts)
    return {"rel": e, **parts}
