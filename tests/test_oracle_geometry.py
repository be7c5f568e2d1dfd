"""Pins for the oracle's geometry and for the shared input layout (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import geometry as G

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("domain,arms", [("cross", 4), ("T", 3), ("L", 2)])
@pytest.mark.parametrize("n", [1, 2, 5, 8, 13])
def test_block_order_is_exactly_the_interior(domain, arms, n):
    """The block listing (arms own the interface lines) partitions the set of
    grid points strictly inside the union of unit squares, found independently
    by cell coverage."""
    listed = G.block_order_points(domain, n)
    assert len(listed) == len(set(listed))
    assert set(listed) == G.interior_points(domain, n)
    assert len(listed) == n * n + arms * n * (n + 1)


def test_unknown_counts_of_the_cross_configs():
    """About 20.5k, 330k and 5.2M unknowns for 64^2, 256^2, 1024^2 blocks."""
    assert W.total_unknowns("cross", 64) == 20736
    assert W.total_unknowns("cross", 256) == 328704
    assert W.total_unknowns("cross", 512) == 1312768
    assert W.total_unknowns("cross", 1024) == 5246976


@pytest.mark.parametrize("domain", ["cross", "T", "L"])
def test_workload_layout_matches_oracle_layout(domain):
    n = 7
    xy = G.node_coordinates(domain, n)
    parts = []
    for b in W.GEOMETRY_BLOCKS[domain]:
        x, y = W.block_coords(b, n)
        parts.append(np.stack([x.ravel(), y.ravel()], axis=1))
    assert np.allclose(np.concatenate(parts), xy, atol=1e-15)


def test_manufactured_solution_vanishes_on_the_edge():
    """p = sin(pi x) sin(pi y) e^{0.3x} is zero on every edge of the cross, so
    the Dirichlet data is homogeneous: check it on the grid points of the
    bounding box that are not unknowns but border one."""
    n = 9
    m = n + 1
    inside = G.interior_points("cross", n)
    for (I, J) in inside:
        for nb in ((I + 1, J), (I - 1, J), (I, J + 1), (I, J - 1)):
            if nb not in inside:
                x, y = nb[0] / m, nb[1] / m
                assert abs(np.sin(np.pi * x) * np.sin(np.pi * y)) < 1e-12


def test_fourier_rhs_is_seeded_and_vanishes_on_block_edges():
    a = W.fourier_rhs("cross", 16, 3)
    b = W.fourier_rhs("cross", 16, 3)
    c = W.fourier_rhs("cross", 16, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.shape == (W.total_unknowns("cross", 16),)
    # an arm's interface line lies on a block edge: f is zero there
    n = 16
    nx, ny = W.block_shape("W", n)
    off = n * n
    wblk = a[off:off + nx * ny].reshape(ny, nx)
    assert np.allclose(wblk[:, -1], 0.0, atol=1e-14)


@pytest.mark.parametrize("geometry", ["cross", "T", "L"])
def test_fourier_rhs_torch_matches_numpy(geometry):
    """The torch evaluation of the seeded workload equals the numpy one."""
    import torch
    a = W.fourier_rhs(geometry, 21, 7)
    b = W.fourier_rhs_torch(geometry, 21, 7, device="cpu").numpy()
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_serving_stream_is_poisson():
    """Exponential gaps with the requested mean; request fields in range."""
    reqs = W.serving_requests(4000, 200.0, seed=0)
    t = np.array([r["arrival_s"] for r in reqs])
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    assert abs(gaps.std() - gaps.mean()) < 0.1 * gaps.mean()  # exponential: std == mean
    assert {r["geometry"] for r in reqs} == {"L", "T", "cross"}
    assert {r["n"] for r in reqs} == {64, 128, 256, 512, 1024}
    assert min(r["nrhs"] for r in reqs) == 1 and max(r["nrhs"] for r in reqs) == 8
