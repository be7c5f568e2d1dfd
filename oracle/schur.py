"""Block structure, Schur complement and Algorithm 1 (oracle; test infrastructure).

Sec. 2.3, Eq. "block_global": in block order the global matrix is
    K = [[A_1, R_12, ...], [R_21, A_2, R_23], ...],   R_ij = R_ji^T,
where each diagonal block A_i is the 5-point operator of block i with its
interfaces treated as Dirichlet.  Here the blocks are read straight off the
assembled K (no second discretisation).  Every layout built here is a star: the
centre C touches every arm and the arms touch only C, so C is the one
"coupled" block and the arms are "independent" (Sec. 2.4, after Alg. 1).

Eq. "Schur_subeq" (read as S_ca = R_ca A_a^{-1} R_ac, the dimensionally
consistent form of the printed S_ij):
    q_a = A_a^{-1} f_a
    (A_c - sum_a S_ca) p_c = f_c - sum_a R_ca q_a  =: f'_c
    p_a = A_a^{-1} (f_a - R_ac p_c)
The block inverses are sparse direct solves -- the plain definition of A^{-1} v.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .geometry import block_ranges
from .krylov import gmres


class BlockSystem:
    """The block pieces of K for one domain."""

    def __init__(self, K: sp.spmatrix, domain: str, n: int, blocks=None):
        """blocks: (name, I0, J0, nx, ny, offset, size) per block in I/O order;
        default: the vertex-centred layout of `domain`."""
        self.K = sp.csr_matrix(K)
        self.domain = domain
        self.n = n
        self.blocks = blocks if blocks is not None else block_ranges(domain, n)
        self.names = [b[0] for b in self.blocks]
        self.sl = {b[0]: slice(b[5], b[5] + b[6]) for b in self.blocks}
        self.arms = [b for b in self.names if b != "C"]
        c = self.sl["C"]
        self.A = {b: sp.csc_matrix(self.K[self.sl[b], self.sl[b]]) for b in self.names}
        self.R_c = {a: sp.csr_matrix(self.K[c, self.sl[a]]) for a in self.arms}   # R_ca
        self.R_a = {a: sp.csr_matrix(self.K[self.sl[a], c]) for a in self.arms}   # R_ac
        self._lu = {b: spla.splu(self.A[b]) for b in self.names}

    def block_solve(self, name: str, v: np.ndarray) -> np.ndarray:
        """A_name^{-1} v (the fast solve's plain definition)."""
        return self._lu[name].solve(np.asarray(v, dtype=np.float64))

    def schur_apply(self, z: np.ndarray) -> np.ndarray:
        """L_c z = A_c z - sum_a R_ca A_a^{-1} R_ac z."""
        w = self.A["C"] @ z
        for a in self.arms:
            w = w - self.R_c[a] @ self.block_solve(a, self.R_a[a] @ z)
        return w

    def schur_dense(self) -> np.ndarray:
        """L_c as a dense matrix (tiny grids only)."""
        Nc = self.n * self.n
        return np.column_stack([self.schur_apply(e) for e in np.eye(Nc)])

    def reduced_rhs(self, f: np.ndarray) -> tuple[np.ndarray, dict]:
        """Alg. 1 steps 1-3: q_a = A_a^{-1} f_a and f'_c = f_c - sum_a R_ca q_a."""
        q = {a: self.block_solve(a, f[self.sl[a]]) for a in self.arms}
        fc = f[self.sl["C"]].copy()
        for a in self.arms:
            fc -= self.R_c[a] @ q[a]
        return fc, q

    def back_substitute(self, f: np.ndarray, pc: np.ndarray) -> np.ndarray:
        """Alg. 1 steps 5-7: p_a = A_a^{-1}(f_a - R_ac p_c); returns the full p."""
        p = np.empty_like(f)
        p[self.sl["C"]] = pc
        for a in self.arms:
            p[self.sl[a]] = self.block_solve(a, f[self.sl[a]] - self.R_a[a] @ pc)
        return p


def algorithm1(bs: BlockSystem, f: np.ndarray, m: int = 30, rtol: float = 1e-10,
               max_iters: int = 3000, precond: str = "A_c", centre_parts=None):
    """Alg. "fft_dd_solver": Schur reduction, preconditioned GMRES on the centre
    block, back substitution.  precond: "A_c" (the paper's A_2^{-1}, applied on
    the right; flexible GMRES), "block_diag" (several coupled blocks stored as
    one centre vector: the exact inverse of each part's own operator, parts given
    as index arrays in `centre_parts`), "jacobi" (inverse diagonal of L_c) or "none".
    The stopping test is taken against ||f||_2 of the whole domain.
    Returns (p, info)."""
    fc, _ = bs.reduced_rhs(f)
    if precond == "A_c":
        M = lambda v: bs.block_solve("C", v)
    elif precond == "block_diag":
        Ac = sp.csc_matrix(bs.A["C"])
        lus = [(ix, spla.splu(sp.csc_matrix(Ac[ix][:, ix]))) for ix in centre_parts]

        def M(v):
            z = np.empty_like(v)
            for ix, lu in lus:
                z[ix] = lu.solve(v[ix])
            return z
    elif precond == "jacobi":
        diag = np.array([bs.schur_apply(e)[i] for i, e in enumerate(np.eye(bs.n * bs.n))]) \
            if bs.n <= 24 else _schur_diagonal(bs)
        M = lambda v: v / diag
    elif precond == "none":
        M = None
    else:
        raise ValueError(precond)
    atol = rtol * float(np.linalg.norm(f))
    pc, info = gmres(bs.schur_apply, fc, m=m, atol=atol, max_iters=max_iters, right_precond=M)
    return bs.back_substitute(f, pc), info


def _schur_diagonal(bs: BlockSystem) -> np.ndarray:
    """diag(L_c) = diag(A_c) - diag(sum_a R_ca A_a^{-1} R_ac), column by column
    only where R is nonzero (the lines next to the arms)."""
    d = bs.A["C"].diagonal().astype(np.float64).copy()
    for a in bs.arms:
        Ra = bs.R_a[a].tocsc()
        cols = np.unique(Ra.nonzero()[1])
        for j in cols:
            e = np.zeros(bs.n * bs.n)
            e[j] = 1.0
            d[j] -= (bs.R_c[a] @ bs.block_solve(a, Ra @ e))[j]
    return d
