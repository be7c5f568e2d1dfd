"""Pins for the oracle's GMRES pieces (CPU only)."""
import numpy as np
import pytest

from oracle import krylov as Kr


def test_mgs_orthonormal_and_matches_qr():
    """Repeated MGS steps give the Q of a QR factorisation (up to signs)."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((8, 50))
    V = A[:1] / np.linalg.norm(A[0])
    Rcols = []
    for j in range(1, 8):
        h, hn, v = Kr.arnoldi_mgs(V, A[j])
        V = np.vstack([V, v])
        Rcols.append((h, hn))
    Q, R = np.linalg.qr(A.T)
    signs = np.sign(np.diag(R))
    assert np.allclose(V, (Q * signs).T, atol=1e-12)
    assert np.allclose(V @ V.T, np.eye(8), atol=1e-13)
    h, hn = Rcols[-1]
    assert np.allclose(np.append(h, hn), (R * signs[:, None])[:, 7], atol=1e-12)


def test_givens_least_squares_matches_lstsq():
    """Givens + back substitution solve min || beta e1 - Hbar y || exactly as a
    library least-squares routine does, and |g_{k}| is its residual norm."""
    rng = np.random.default_rng(1)
    m = 9
    Hbar = np.triu(rng.standard_normal((m + 1, m)), -1)
    beta = 2.5
    cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
    g[0] = beta
    R = np.zeros((m + 1, m))
    for j in range(m):
        col = Hbar[: j + 2, j].copy()
        res = Kr.givens_step(col, cs, sn, g, j)
        R[: j + 2, j] = col
        y = Kr.back_substitute(R, g, j + 1)
        rhs = np.zeros(j + 2)
        rhs[0] = beta
        y_ref, *_ = np.linalg.lstsq(Hbar[: j + 2, : j + 1], rhs, rcond=None)
        assert np.allclose(y, y_ref, rtol=1e-10, atol=1e-12)
        assert abs(res - np.linalg.norm(rhs - Hbar[: j + 2, : j + 1] @ y_ref)) < 1e-10


def test_gmres_exact_in_N_steps_and_restarted():
    rng = np.random.default_rng(2)
    N = 30
    A = rng.standard_normal((N, N)) + N * np.eye(N)
    b = rng.standard_normal(N)
    x_ref = np.linalg.solve(A, b)
    x, info = Kr.gmres(lambda v: A @ v, b, m=N, atol=1e-13 * np.linalg.norm(b))
    assert np.allclose(x, x_ref, rtol=1e-11)
    x2, info2 = Kr.gmres(lambda v: A @ v, b, m=5, atol=1e-12 * np.linalg.norm(b), max_iters=500)
    assert info2["restarts"] > 1 and np.allclose(x2, x_ref, rtol=1e-9)
    # flexible GMRES with a right preconditioner reaches the same solution
    M = np.linalg.inv(A + 0.1 * rng.standard_normal((N, N)))
    x3, info3 = Kr.gmres(lambda v: A @ v, b, m=10, atol=1e-12 * np.linalg.norm(b),
                         right_precond=lambda v: M @ v)
    assert np.allclose(x3, x_ref, rtol=1e-9) and info3["iterations"] < info2["iterations"]


def test_gmres_history_is_the_minimal_residual_over_the_krylov_space():
    """The GMRES residual after k steps is min ||b - A x|| over x in K_k(A, b)
    (the defining property), found here by least squares over the explicit
    Krylov power basis; with a fixed right preconditioner M it is the same over
    x in M K_k(A M, b)."""
    rng = np.random.default_rng(7)
    N = 40
    A = rng.standard_normal((N, N)) / np.sqrt(N) + 2.0 * np.eye(N)
    b = rng.standard_normal(N)
    M = np.linalg.inv(A + 0.3 * rng.standard_normal((N, N)) / np.sqrt(N))
    for precond in (None, M):
        Aop = A if precond is None else A @ precond
        _, info = Kr.gmres(lambda v: A @ v, b, m=12, atol=0.0, max_iters=8,
                           right_precond=None if precond is None else (lambda v: precond @ v))
        hist = info["history"]
        P = np.zeros((N, 8))
        v = b.copy()
        for k in range(8):
            P[:, k] = v / np.linalg.norm(v)
            v = Aop @ P[:, k]
        for k in range(1, 9):
            Q, _ = np.linalg.qr(P[:, :k])          # an orthonormal basis of K_k
            y, *_ = np.linalg.lstsq(Aop @ Q, b, rcond=None)
            best = np.linalg.norm(b - Aop @ Q @ y)
            assert abs(hist[k] - best) <= 1e-10 * np.linalg.norm(b), (precond is None, k, hist[k], best)
