"""Direct solve p = K^{-1} b (oracle; test infrastructure).

The paper's method reaches the exact solution of the discrete system (Sec. 2.3:
the Schur elimination is exact; GMRES is run to a tolerance), so the plain
definition of its result is the solution of K p = b.  Tiny systems use dense LU
(numpy), larger ones a sparse LU (SciPy's SuperLU); both are library primitives
used as one step.
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
            self._lu = spla.splu(sp.csc_matrix(K), permc_spec="COLAMD")

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
