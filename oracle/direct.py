"""Direct solve p = K^{-1} b (oracle; test infrastructure).

The paper's method reaches the exact solution of the discrete system (Sec. 2.3:
the Schur elimination is exact; GMRES is run to a tolerance), so the plain
definition of its result is the solution of K p = b.  Tiny systems use dense LU
(numpy), larger ones a sparse LU (SciPy's SuperLU); both are library primitives
used as one step.  A second route written here from its textbook definition,
conjugate gradients on -K (symmetric positive definite for kappa <= 0; Sec. 2.1
makes K the symmetric 5-point operator), cross-checks the library solves.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DENSE_LIMIT = 3000


class Factor:
    """A factorisation of K that can be reused for several right-hand sides."""

    def __init__(self, K: sp.spmatrix):
        self.N = K.shape[0]
        if self.N <= DENSE_LIMIT:
            self._dense = np.asarray(K.todense())
            self._lu = None
        else:
            self._dense = None
            # minimum degree on the structure of K + K^T: K is symmetric, and on
            # a 5-point grid this ordering keeps half the fill of COLAMD (5.2M
            # unknowns factor in about a minute).  The ordering is a permutation
            # and does not change what is solved.
            self._lu = spla.splu(sp.csc_matrix(K), permc_spec="MMD_AT_PLUS_A")

    def solve(self, b: np.ndarray) -> np.ndarray:
        if self._dense is not None:
            if b.ndim == 1:
                return np.linalg.solve(self._dense, b)
            return np.linalg.solve(self._dense, b.T).T.copy()
        if b.ndim == 1:
            return self._lu.solve(b)
        return self._lu.solve(np.asfortranarray(b.T)).T.copy()


def solve(K: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """p = K^{-1} b; b may be (N,) or (nrhs, N)."""
    return Factor(K).solve(b)


def conjugate_gradient(K: sp.spmatrix, b: np.ndarray, rtol: float = 1e-12, max_iters: int | None = None):
    """p = K^{-1} b by plain conjugate gradients on A = -K (SPD), x0 = 0, stopping
    when the residual norm falls to rtol ||b||_2 or after max_iters (default 20 N)
    steps; every 50 steps the updated residual is replaced by b - K p, so the
    test is taken on the true residual up to the last 50 steps' drift.
    Returns (p, steps)."""
    A = -sp.csr_matrix(K)
    rhs = -np.asarray(b, dtype=np.float64)
    N = rhs.shape[0]
    if max_iters is None:
        max_iters = 20 * N
    x = np.zeros(N)
    r = rhs.copy()
    d = r.copy()
    rr = float(r @ r)
    target = (rtol * float(np.linalg.norm(rhs))) ** 2
    steps = 0
    while rr > target and steps < max_iters:
        Ad = A @ d
        alpha = rr / float(d @ Ad)
        x += alpha * d
        r -= alpha * Ad
        steps += 1
        if steps % 50 == 0:          # replace the recurrence by the true residual
            r = rhs - A @ x
        rr_new = float(r @ r)
        d = r + (rr_new / rr) * d
        rr = rr_new
    return x, steps
