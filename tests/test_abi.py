"""The C-ABI library builds, loads and exports every entry point include/fpg.h
declares; descriptor validation and workspace sizing need no GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_2509_23180_gb300 import binding as B
from paper_2509_23180_gb300 import build as Bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return B.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fpg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fpg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(B.EXPORTED)


def test_status_strings_and_version(lib):
    assert lib.fpg_version().startswith(b"fpg")
    for s in range(8):
        assert lib.fpg_status_string(s).startswith(b"FPG_")


@pytest.mark.parametrize("geom,arms", [("cross", 4), ("T", 3), ("L", 2)])
def test_unknowns_and_workspace(lib, geom, arms):
    d = B.make_desc(geom, 64, 0.0, nrhs=2)
    assert B.unknowns(d) == 64 * 64 + arms * 64 * 65
    ws = B.workspace_bytes(d)
    # at least V (m+1 vectors), Z (m), f and a temporary per right-hand side
    assert ws > 8 * 2 * (61 * 64 * 64 + 2 * B.unknowns(d))


@pytest.mark.parametrize("field,value", [("n", 1), ("n", 5000), ("kappa", 1.0), ("nrhs", 0), ("restart", 0),
                                         ("restart", 500), ("rtol", 0.0), ("rtol", 1.0),
                                         ("precond_precision", 16), ("schur_mode", 7), ("geometry", 3),
                                         ("max_iters", 0), ("boundary", 2), ("boundary", -1)])
def test_invalid_descriptors_rejected(lib, field, value):
    d = B.make_desc("cross", 16)
    setattr(d, field, value)
    with pytest.raises(B.FpgError) as e:
        B.workspace_bytes(d)
    assert e.value.status == B.FPG_EINVAL


def test_create_rejects_small_workspace_without_touching_gpu(lib):
    import ctypes
    d = B.make_desc("cross", 16)
    h = ctypes.c_void_p()
    # a dummy non-null address: the size check fails before any CUDA call
    st = lib.fpg_create_domain(ctypes.byref(d), 0x1000, 16, None, ctypes.byref(h))
    assert st == B.FPG_ENOMEM and not h.value


def test_neumann_sided_cross_descriptor(lib):
    """Sec. 3.1 boundary pattern: 5 n^2 unknowns on the cell-centred cross; other
    geometries and lengths without a DCT-II plan are refused as unsupported."""
    d = B.make_desc("cross", 64, -10.0, nrhs=2, boundary="neumann_sides")
    assert B.unknowns(d) == 5 * 64 * 64
    assert B.workspace_bytes(d) > 8 * 2 * (31 * 64 * 64 + 2 * B.unknowns(d))
    for geom, n in (("T", 64), ("L", 64), ("cross", 63), ("cross", 34), ("cross", 4096)):
        bad = B.make_desc(geom, n, boundary="neumann_sides")
        with pytest.raises(B.FpgError) as e:
            B.workspace_bytes(bad)
        assert e.value.status == B.FPG_EUNSUPPORTED, (geom, n)


@pytest.mark.parametrize("kind,nt,ns,want", [(0, 64, 40, "OK"), (0, 4097, 8, "EINVAL"), (1, 64, 8, "OK"),
                                             (1, 63, 8, "EINVAL"), (1, 34, 8, "EUNSUPPORTED"),
                                             (1, 4096, 8, "EINVAL"), (2, 45, 8, "OK"), (2, 17, 8, "EUNSUPPORTED"),
                                             (2, 1, 8, "EINVAL"), (3, 64, 8, "EINVAL"), (0, 64, 0, "EINVAL")])
def test_rect_plan_bytes(lib, kind, nt, ns, want):
    nb = ctypes.c_size_t()
    st = lib.fpg_rect_plan_bytes(kind, nt, ns, 2, ctypes.byref(nb))
    assert st == getattr(B, "FPG_" + want)
    if want == "OK":
        assert nb.value >= 2 * 8 * nt * ns + 2 * 8 * nt * ns  # pivots + scratch of two rectangles


def test_chain_descriptor(lib):
    """Several coupled blocks: a chain of K crosses has (2K-1)(n+1)-1 by n row
    unknowns plus 2K + 2 arms; K outside 2..5, a chain count on another geometry,
    and the literal Schur form or Neumann sides on a chain are refused."""
    n = 16
    for K in (2, 3, 5):
        d = B.make_desc("chain", n, 0.0, chain=K)
        assert B.unknowns(d) == ((2 * K - 1) * (n + 1) - 1) * n + (2 * K + 2) * n * (n + 1)
    for kw, want in (({"chain": 1}, B.FPG_EINVAL), ({"chain": 6}, B.FPG_EINVAL),
                     ({"chain": 2, "schur_mode": "literal"}, B.FPG_EUNSUPPORTED),
                     ({"chain": 2, "boundary": "neumann_sides"}, B.FPG_EUNSUPPORTED)):
        with pytest.raises(B.FpgError) as e:
            B.workspace_bytes(B.make_desc("chain", n, 0.0, **kw))
        assert e.value.status == want, kw
    with pytest.raises(B.FpgError) as e:
        B.workspace_bytes(B.make_desc("cross", n, 0.0, chain=2))
    assert e.value.status == B.FPG_EINVAL


def test_batch_create_arguments(lib):
    """The batch runtime's descriptor checks need no device."""
    h = ctypes.c_void_p()
    for slots, maxd, per, busy in ((0, 4, 0, 0), (65, 4, 0, 0), (8, 0, 0, 0), (8, 257, 0, 0), (8, 4, 17, 0),
                                   (8, 4, -1, 0), (8, 4, 0, -1)):
        d = B.BatchDescC(slots, maxd, per, busy)
        assert lib.fpg_batch_create(ctypes.byref(d), ctypes.c_void_p(4096), 1 << 20, ctypes.byref(h)) == B.FPG_EINVAL
