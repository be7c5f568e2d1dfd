"""GPU parity of the size-specialised line DST kernels (fast solve, a1) and of
the integer-pipe FP64 <-> FP32 conversions of the mixed-precision path.

The specialised kernels cover p = n + 1 = 65, 257 (Rader), 513 in FP64 and
also 1025 in FP32; every other length runs the generic FFT engine, which the
tests use as a second, independent GPU path (FPG_OPT_DST_ENGINE = 1).
"""
import numpy as np
import pytest

import workloads as W
from tests.parity import assert_solution, rel  # noqa: F401
from oracle import operator as O
from oracle import schur as S
from oracle import transforms as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




def mode_mix(n, kappa, seed, count=2):
    """Random combinations of rectangle eigenmodes and their exact A^{-1} images
    (A^{-1} q_kl = q_kl / lambda_kl, Sec. 2.1)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n + 1)
    ks = [(1, 1), (n, n), (n // 2, 3), (7, n - 1), (2, 2), (n - 3, n // 3 + 1)]
    v = np.zeros((count, n * n))
    want = np.zeros((count, n * n))
    for k, l in ks:
        q = T.rectangle_mode(k, l, n, n)
        lam = T.rectangle_eigenvalue(k, l, n, n, h, kappa)
        c = rng.standard_normal(count)
        v += c[:, None] * q[None, :]
        want += (c / lam)[:, None] * q[None, :]
    return v, want


@pytest.mark.parametrize("n", [64, 256, 512, 1024])
def test_line_dst_fp32_modes_no_worse_than_generic(lib, n):
    """FP32 preconditioner through the specialised kernels reproduces the closed
    form of a mode mixture as accurately as the generic FFT engine does."""
    from paper_2509_23180_gb300 import binding as B
    kappa = -10.0
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=2, precond_precision=32))
    assert d.fast_solve_path() == 1
    v, want = mode_mix(n, kappa, seed=n)
    z = torch.zeros((2, n * n), dtype=torch.float32, device="cuda")
    d.apply_precond(dev(v), z, 2)
    err_s = rel(host(z), want)
    d.set_option(B.OPT_DST_ENGINE, 1)
    assert d.fast_solve_path() == 0
    zg = torch.zeros_like(z)
    d.apply_precond(dev(v), zg, 2)
    err_g = rel(host(zg), want)
    d.close()
    assert err_s < 1e-4 and err_s <= 2.0 * err_g + 1e-7, (err_s, err_g)


@pytest.mark.parametrize("n", [64, 256, 512])
def test_line_dst_fp64_random_matches_generic(lib, n):
    """FP64: specialised and generic engines agree on random vectors (all modes
    present) to rounding, on the centre block and on both arm layouts."""
    from paper_2509_23180_gb300 import binding as B
    kappa = 0.0
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=3))
    d.set_option(B.OPT_DST_ENGINE, 2)
    assert d.fast_solve_path() == 1
    outs = {}
    for engine in (2, 1):
        d.set_option(B.OPT_DST_ENGINE, engine)
        for blk, name in ((0, "C"), (1, "W"), (4, "N")):
            nx, ny = W.block_shape(name, n)
            v = W.random_block_vectors(3, nx * ny, seed=blk + 7)
            z = torch.zeros_like(dev(v))
            d.block_solve(blk, dev(v), z, 3)
            outs[(engine, name)] = host(z)
    d.close()
    for name in ("C", "W", "N"):
        assert rel(outs[(2, name)], outs[(1, name)]) < 1e-12, name


@pytest.mark.parametrize("prec,tol", [(64, 1e-11), (32, 5e-5)])
def test_line_dst_vs_oracle_n256(lib, prec, tol):
    """a1 on the bench block size against the oracle's direct block solve."""
    from paper_2509_23180_gb300 import binding as B
    n, kappa = 256, -10.0
    bs = S.BlockSystem(O.assemble("cross", n, kappa), "cross", n)
    d = B.Domain(B.make_desc("cross", n, kappa, nrhs=2, precond_precision=prec))
    d.set_option(B.OPT_DST_ENGINE, 2)
    assert d.fast_solve_path() == 1
    v = W.random_block_vectors(2, n * n, seed=3)
    z = torch.zeros((2, n * n), dtype=torch.float64 if prec == 64 else torch.float32, device="cuda")
    d.apply_precond(dev(v), z, 2)
    d.close()
    want = np.stack([bs.block_solve("C", vi) for vi in v])
    assert rel(host(z), want) < tol


def test_line_dst_engine_choice(lib):
    """Default choice: FP32 always specialised where compiled; FP64 only when the
    batch gives enough threads (10 x 256^2 does, one 64^2 block does not)."""
    from paper_2509_23180_gb300 import binding as B
    for prec, n, nrhs, want in ((32, 256, 2, 1), (64, 256, 10, 1), (64, 256, 64, 1), (64, 64, 1, 0)):
        d = B.Domain(B.make_desc("cross", n, 0.0, nrhs=nrhs, restart=2, precond_precision=prec))
        assert d.fast_solve_path() == want, (prec, n, nrhs)
        d.close()


def test_line_dst_ragged_tiles_match_generic(lib):
    """Ragged line tiles (the S arm has n + 1 lines of contiguous rows) give the
    generic engine's result."""
    from paper_2509_23180_gb300 import binding as B
    n = 64
    d = B.Domain(B.make_desc("cross", n, -3.0, nrhs=4))
    d.set_option(B.OPT_DST_ENGINE, 2)
    nx, ny = W.block_shape("S", n)
    v = W.random_block_vectors(4, nx * ny, seed=11)
    z = torch.zeros_like(dev(v))
    d.block_solve(3, dev(v), z, 4)
    d.set_option(B.OPT_DST_ENGINE, 1)
    zg = torch.zeros_like(z)
    d.block_solve(3, dev(v), zg, 4)
    d.close()
    assert rel(host(z), host(zg)) < 1e-12


def _f32_bits(t):
    return host(t.view(torch.int32))


def test_convert_f64_to_f32_rounding(lib):
    """Round to nearest even on the IEEE-754 encodings equals the hardware
    conversion in the binary32 normal range, ties and binade edges included."""
    from paper_2509_23180_gb300 import binding as B
    rng = np.random.default_rng(0)
    x = [rng.standard_normal(20000) * np.exp2(rng.integers(-120, 120, 20000))]
    f = rng.standard_normal(5000).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + nxt.astype(np.float64)) / 2  # exact ties
    x += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)]
    edges = np.array([np.finfo(np.float32).max, -np.finfo(np.float32).max, 2.0 ** -126, -(2.0 ** -126),
                      2.0 ** 127 * (2 - 2.0 ** -24) * (1 - 2.0 ** -40), 1.0, -1.0, 0.0, 3.0 * 2.0 ** -127])
    x.append(edges)
    x = np.concatenate(x)
    xd = dev(x)
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    B.convert(xd, out)
    ref = xd.float()
    normal = (np.abs(x) >= 2.0 ** -126) & (np.abs(x) < 2.0 ** 127 * (2 - 2.0 ** -24))
    assert np.array_equal(_f32_bits(out)[normal], _f32_bits(ref)[normal])
    got = host(out)
    tiny = np.abs(x) < 2.0 ** -126
    assert np.all(got[tiny] == 0.0) and np.array_equal(np.signbit(got[tiny]), np.signbit(x[tiny]))
    neg0 = torch.tensor([-0.0], dtype=torch.float64, device="cuda")
    o = torch.empty(1, dtype=torch.float32, device="cuda")
    B.convert(neg0, o)
    assert np.signbit(host(o)[0]) and host(o)[0] == 0.0
    big = dev(np.array([2.0 ** 128, -(2.0 ** 130), np.inf]))
    ob = torch.empty(3, dtype=torch.float32, device="cuda")
    B.convert(big, ob)
    assert np.array_equal(host(ob), np.array([np.inf, -np.inf, np.inf], dtype=np.float32))


def test_convert_f32_to_f64_exact(lib):
    from paper_2509_23180_gb300 import binding as B
    rng = np.random.default_rng(1)
    f = (rng.standard_normal(20000) * np.exp2(rng.integers(-120, 120, 20000))).astype(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, np.finfo(np.float32).max,
                                     np.finfo(np.float32).tiny], dtype=np.float32)])
    fd = dev(f, torch.float32)
    out = torch.empty(f.size, dtype=torch.float64, device="cuda")
    B.convert(fd, out)
    got, want = host(out), f.astype(np.float64)
    sub = (f != 0) & (np.abs(f) < np.finfo(np.float32).tiny)  # binary32 subnormals
    assert np.array_equal(got[~sub], want[~sub])
    assert np.all(got[sub] == 0.0)
    assert np.array_equal(np.signbit(got), np.signbit(f))
    sd = dev(np.array([1e-40, -1e-41], dtype=np.float32), torch.float32)
    os_ = torch.empty(2, dtype=torch.float64, device="cuda")
    B.convert(sd, os_)
    g2 = host(os_)
    assert np.all(g2 == 0.0) and np.array_equal(np.signbit(g2), [False, True])


@pytest.mark.parametrize("geom,n,kappa", [("cross", 64, 0.0), ("T", 64, -10.0), ("L", 256, 0.0),
                                          ("cross", 256, -10.0)])
def test_schur_transform_form_vs_oracle(lib, geom, n, kappa):
    """a2 with the reduced interface term applied as delta^2 Q diag(g_k) Q by two
    DST-I per line: equal to the oracle's Schur matvec (exact arm solves) and to
    the O(n^2) Toeplitz-minus-Hankel sum, for FP64 and FP32 z."""
    from paper_2509_23180_gb300 import binding as B
    bs = S.BlockSystem(O.assemble(geom, n, kappa), geom, n)
    d = B.Domain(B.make_desc(geom, n, kappa, nrhs=3))
    d.set_option(B.OPT_SCHUR_TRANSFORM, 1)
    zv = W.random_block_vectors(3, n * n, seed=n + 1)
    w = torch.zeros((3, n * n), dtype=torch.float64, device="cuda")
    d.apply_schur(dev(zv), 64, w, 3)
    got = host(w)
    want = np.stack([bs.schur_apply(zi) for zi in zv])
    assert rel(got, want) < 1e-11
    d.set_option(B.OPT_SCHUR_TRANSFORM, 0)  # the O(n^2) table sum
    wd = torch.zeros_like(w)
    d.apply_schur(dev(zv), 64, wd, 3)
    assert rel(host(wd), want) < 1e-11
    assert rel(got, host(wd)) < 1e-13
    d.set_option(B.OPT_SCHUR_TRANSFORM, 1)
    z32 = torch.as_tensor(zv, dtype=torch.float32, device="cuda")
    d.apply_schur(z32, 32, w, 3)
    want32 = np.stack([bs.schur_apply(zi) for zi in zv.astype(np.float32).astype(np.float64)])
    d.close()
    assert rel(host(w), want32) < 1e-11


@pytest.mark.parametrize("n", [64, 256, 512, 1024])
def test_bulk_copy_forward_dst_is_bit_identical(lib, n):
    """The persistent forward DST with bulk asynchronous row copies computes
    exactly what the one-CTA-per-tile kernel does (FP32 preconditioner, and a
    whole FP32-preconditioned solve with right-hand sides dropping out)."""
    from paper_2509_23180_gb300 import binding as B
    d = B.Domain(B.make_desc("cross", n, -10.0, nrhs=3, restart=20, rtol=1e-10, precond_precision=32))
    v = dev(W.random_block_vectors(3, n * n, seed=n + 5))
    outs = []
    for bulk in (0, 1):
        d.set_option(B.OPT_DST_BULK, bulk)
        z = torch.zeros((3, n * n), dtype=torch.float32, device="cuda")
        d.apply_precond(v, z, 3)
        outs.append(host(z))
    assert np.array_equal(outs[0], outs[1])
    if n <= 256:
        f = dev(W.rhs_batch("cross", n, [1, 2, 3], kind="fourier"))
        sols = []
        for bulk in (0, 1):
            d.set_option(B.OPT_DST_BULK, bulk)
            d.set_rhs(f)
            p = torch.zeros_like(f)
            assert d.solve(p)[0] == B.FPG_OK
            sols.append(host(p))
        assert np.array_equal(sols[0], sols[1])
    d.close()
