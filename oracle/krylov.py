"""Restarted (flexible) GMRES, step by step (oracle; test infrastructure).

Sec. 2.4 lists the GMRES steps: build a Krylov basis, orthonormalise it by
Gram-Schmidt into V_d, solve min || ||r0|| e_1 - Hbar_d y ||_2 over the Hessenberg
matrix of the Arnoldi process, update p += V_d y, stop once the residual is
below the tolerance, else restart.  The reading used here (the paper builds a
power basis first and orthonormalises it afterwards) is the standard Arnoldi
process: each new vector is orthogonalised immediately, with modified
Gram-Schmidt.  The least-squares problem is solved with Givens rotations, and
|g_{j+1}| is the residual norm of the current iterate.

The FFT preconditioner A_2^{-1} (Eqs. "precond_iter"-"precond_basis_equ") is
applied on the right, as the text says; with a right preconditioner M the basis
is built for L M and the update is p += Z y with Z = [M v_1, ..., M v_d]
(flexible GMRES, which also allows M to change from step to step).
"""
from __future__ import annotations

import math

import numpy as np


def arnoldi_mgs(V: np.ndarray, w: np.ndarray):
    """One modified Gram-Schmidt step: orthogonalise w against the rows of V
    one after another.  Returns (h[0..j], h_{j+1,j}, v_{j+1})."""
    w = np.array(w, dtype=np.float64, copy=True)
    h = np.zeros(V.shape[0])
    for i in range(V.shape[0]):
        h[i] = float(np.dot(w, V[i]))
        w -= h[i] * V[i]
    hn = float(np.linalg.norm(w))
    return h, hn, (w / hn if hn > 0 else w)


def givens_step(Hcol: np.ndarray, cs: np.ndarray, sn: np.ndarray, g: np.ndarray, j: int):
    """Bring column j of Hbar (length j+2) to triangular form.

    Apply the j earlier rotations, then form the rotation (c, s) that zeroes
    entry j+1:  c = h_j / r, s = h_{j+1} / r, r = sqrt(h_j^2 + h_{j+1}^2), and
    apply it to g.  Updates Hcol, cs, sn, g in place; returns |g_{j+1}|."""
    for i in range(j):
        a, b = Hcol[i], Hcol[i + 1]
        Hcol[i] = cs[i] * a + sn[i] * b
        Hcol[i + 1] = -sn[i] * a + cs[i] * b
    a, b = Hcol[j], Hcol[j + 1]
    r = math.hypot(a, b)
    c, s = (1.0, 0.0) if r == 0.0 else (a / r, b / r)
    cs[j], sn[j] = c, s
    Hcol[j] = r
    Hcol[j + 1] = 0.0
    g[j + 1] = -s * g[j]
    g[j] = c * g[j]
    return abs(g[j + 1])


def back_substitute(R: np.ndarray, g: np.ndarray, k: int) -> np.ndarray:
    """Solve the k x k upper-triangular system R[:k,:k] y = g[:k]."""
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(R[i, i + 1:k], y[i + 1:k])) / R[i, i]
    return y


def gmres(apply_A, b: np.ndarray, m: int = 30, atol: float = 1e-10, max_iters: int = 3000,
          right_precond=None, x0: np.ndarray | None = None):
    """Restarted GMRES(m) for A x = b, stopping when ||b - A x||_2 <= atol.

    right_precond: None (plain GMRES) or a callable v -> M v (flexible GMRES).
    Returns (x, info) with info = {iterations, restarts, history, converged,
    true_residual}."""
    N = b.shape[0]
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    history = []
    total = 0
    restarts = 0
    converged = False
    while total < max_iters:
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
        history.append(beta)
        if beta <= atol:
            converged = True
            break
        V = np.zeros((m + 1, N))
        Z = np.zeros((m, N)) if right_precond is not None else None
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            z = right_precond(V[j]) if right_precond is not None else V[j]
            if Z is not None:
                Z[j] = z
            w = apply_A(z)
            h, hn, vn = arnoldi_mgs(V[: j + 1], w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            V[j + 1] = vn
            col = H[: j + 2, j].copy()
            res = givens_step(col, cs, sn, g, j)
            H[: j + 2, j] = col
            total += 1
            k = j + 1
            history.append(res)
            if res <= atol or hn == 0.0 or total >= max_iters:
                break
        y = back_substitute(H, g, k)
        basis = Z if Z is not None else V
        x = x + y @ basis[:k]
        restarts += 1
    r = b - apply_A(x)
    true_res = float(np.linalg.norm(r))
    converged = converged or true_res <= atol
    return x, {"iterations": total, "restarts": restarts, "history": history,
               "converged": converged, "true_residual": true_res}
