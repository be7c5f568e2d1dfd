"""Cross with Neumann arm sides (oracle; test infrastructure -- only tests/,
smoke() and bench.py's reference leg use it).

The boundary conditions of the paper's precision validation (Sec. 3.1, Eq.
"cross_equation"): zero Dirichlet at the four far ends of the cross, zero
normal derivative on the sides of the arms.  Here on the cross of unit
squares C = [0,1]^2, W = [-1,0]x[0,1], E = [1,2]x[0,1], S = [0,1]x[-1,0],
N = [0,1]x[1,2]: Dirichlet on x = -1, x = 2, y = -1, y = 2; Neumann on the
edges y = 0, 1 of W and E and x = 0, 1 of S and N.

Grid: cell-centred with h = 1/n (the Neumann edges sit half a cell from the
unknowns, as in the matrix of Eq. "submat_Neumann", whose corner rows lose one
delta).  An unknown sits at every cell centre ((I+1/2)h, (J+1/2)h) inside the
cross, so every block is n x n.  At a boundary face the ghost value beyond it
is the cell's own value for a Neumann face (the row loses one delta) and minus
the cell's value for a Dirichlet face (zero at the face by linear
interpolation; the row gains -delta).  The operator is assembled here from
cell membership and face position alone, with no block structure.

Block order (the library's I/O convention): C, W, E, S, N, each row-major with
x fastest.

The analytic solution follows the paper's construction (Eqs.
"cross_analytical_solultion", "cross_ana_sol_psi"): p = sin(psi(x)) sin(psi(y))
with a cubic psi that is 0 (mod pi) at the Dirichlet ends and pi/2 (mod pi) on
the Neumann lines, so that cos(psi) psi' = 0 there:
    psi(-1) = 0, psi(0) = pi/2, psi(1) = 3 pi/2, psi(2) = 2 pi
    psi(t) = (t + 1) [pi/2 + (pi/4) t - (pi/6) t (t - 1)]   (Newton form).
The paper's own constants give psi(7L) = pi/2, which contradicts its Dirichlet
condition at x = 7L and y = 7L; its block sizes live in a lost figure.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

BLOCKS = ("C", "W", "E", "S", "N")


def _block_cells(n: int) -> dict:
    """Integer cell range of every block: (I0, J0) of its first cell."""
    return {"C": (0, 0), "W": (-n, 0), "E": (n, 0), "S": (0, -n), "N": (0, n)}


def inside(I: int, J: int, n: int) -> bool:
    """Is the cell [I h, (I+1) h] x [J h, (J+1) h] inside the cross?"""
    in_band_x = 0 <= I < n
    in_band_y = 0 <= J < n
    return (in_band_y and -n <= I < 2 * n) or (in_band_x and -n <= J < 2 * n)


def block_ranges(n: int) -> list[tuple[str, int, int, int, int, int, int]]:
    """Per block in I/O order: (name, I_first, J_first, nx, ny, offset, size)."""
    out, off = [], 0
    for b, (i0, j0) in _block_cells(n).items():
        out.append((b, i0, j0, n, n, off, n * n))
        off += n * n
    return out


def cells(n: int) -> list[tuple[int, int]]:
    """The unknowns (cell indices) in block order."""
    pts = []
    for _, i0, j0, nx, ny, _, _ in block_ranges(n):
        for j in range(ny):
            for i in range(nx):
                pts.append((i0 + i, j0 + j))
    return pts


def coordinates(n: int) -> np.ndarray:
    """Cell centres (x, y) in block order, shape (5 n^2, 2)."""
    return (np.asarray(cells(n), dtype=np.float64) + 0.5) / n


def face_kind(I: int, J: int, di: int, dj: int, n: int) -> str:
    """Kind of the face between the inside cell (I, J) and its outside neighbour
    (I+di, J+dj): "dirichlet" on the far ends x = -1, 2 and y = -1, 2,
    "neumann" on every other edge of the cross."""
    x_face = I + (di > 0)  # face position in units of h, for a step along x
    y_face = J + (dj > 0)
    if di != 0 and x_face in (-n, 2 * n):
        return "dirichlet"
    if dj != 0 and y_face in (-n, 2 * n):
        return "dirichlet"
    return "neumann"


def assemble(n: int, kappa: float = 0.0) -> sp.csr_matrix:
    """K over all 5 n^2 unknowns, rows/columns in block order."""
    pts = cells(n)
    index = {p: k for k, p in enumerate(pts)}
    d = float(n) ** 2
    rows, cols, vals = [], [], []
    for k, (I, J) in enumerate(pts):
        diag = -4.0 * d + kappa
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            q = index.get((I + di, J + dj))
            if q is not None:
                rows.append(k)
                cols.append(q)
                vals.append(d)
            elif face_kind(I, J, di, dj, n) == "neumann":
                diag += d   # ghost = the cell's value
            else:
                diag -= d   # ghost = minus the cell's value
        rows.append(k)
        cols.append(k)
        vals.append(diag)
    N = len(pts)
    return sp.csr_matrix((np.asarray(vals), (np.asarray(rows), np.asarray(cols))), shape=(N, N))


# ---- analytic solution -------------------------------------------------------

def _psi_coeffs():
    """Monomial coefficients (a0, a1, a2, a3) of psi: expanding
    (t + 1)(b0 + b1 t + b2 t^2) with b0 = pi/2, b1 = pi/4 + pi/6, b2 = -pi/6."""
    b0, b1, b2 = np.pi / 2, np.pi / 4 + np.pi / 6, -np.pi / 6
    return b0, b0 + b1, b1 + b2, b2


def psi(t):
    t = np.asarray(t, dtype=np.float64)
    return (t + 1.0) * (np.pi / 2 + (np.pi / 4) * t - (np.pi / 6) * t * (t - 1.0))


def dpsi(t):
    t = np.asarray(t, dtype=np.float64)
    _, a1, a2, a3 = _psi_coeffs()
    return a1 + 2.0 * a2 * t + 3.0 * a3 * t * t


def d2psi(t):
    t = np.asarray(t, dtype=np.float64)
    _, _, a2, a3 = _psi_coeffs()
    return 2.0 * a2 + 6.0 * a3 * t


def exact(x, y):
    return np.sin(psi(x)) * np.sin(psi(y))


def source(x, y, kappa: float = 0.0):
    """f = lap p + kappa p for the analytic p."""
    def s2(t):  # d^2/dt^2 sin(psi(t))
        return -np.sin(psi(t)) * dpsi(t) ** 2 + np.cos(psi(t)) * d2psi(t)
    return s2(x) * np.sin(psi(y)) + np.sin(psi(x)) * s2(y) + kappa * exact(x, y)


def manufactured(n: int, kappa: float = 0.0):
    """(p, f) of the analytic solution at the cell centres, block order."""
    xy = coordinates(n)
    return exact(xy[:, 0], xy[:, 1]), source(xy[:, 0], xy[:, 1], kappa)
