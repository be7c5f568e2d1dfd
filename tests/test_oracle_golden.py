"""The stored expected values still equal what the oracle computes (CPU only)."""
import os

import numpy as np
import pytest

from tests.golden.make_golden import CASES, EXTRA_CASES, HERE, expected, expected_extra


def load_golden(fname):
    with open(os.path.join(HERE, fname)) as fh:
        return np.array([float(l) for l in fh if not l.startswith("#")])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_golden_matches_oracle(case):
    fname, domain, n, kappa, kind, seed = case
    _, p = expected(domain, n, kappa, kind, seed)
    g = load_golden(fname)
    assert g.shape == p.shape
    assert np.allclose(g, p, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("case", EXTRA_CASES, ids=[c[0] for c in EXTRA_CASES])
def test_extra_golden_matches_oracle(case):
    fname, geometry, n, kappa, extra = case
    _, p = expected_extra(geometry, n, kappa, extra)
    g = load_golden(fname)
    assert g.shape == p.shape
    assert np.allclose(g, p, rtol=1e-13, atol=1e-16)
