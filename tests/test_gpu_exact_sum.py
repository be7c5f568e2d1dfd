"""The Arnoldi step's projections are exact sums (csrc/fpg_exactsum.cuh): h_{0,0} =
(w, v_0) of Alg. 2's modified Gram-Schmidt equals the correctly rounded value of the
exact dot product whenever each thread's own partial is exact and a multiple of
2^-62 of the largest partial (the fixed-point grid of the sum), whatever the order in
which the partials meet.

The inputs put one nonzero element of w in each of a few threads (consecutive
indices land in different threads for every launch shape), with v_0 = 2^-6 on every
element of a vector of 4096 (unit norm, exact products).  The partials then are the
w_i 2^-6 themselves, and the cases are chosen where a floating-point tree depends on
its order: a cancellation of +-2^54 around small terms, and a sum on a rounding tie
of binary64 pushed just above it by a term 2^-8.  The expected values are exact
rational arithmetic rounded once to binary64 (Python's Fraction and float).
"""
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEN = 4096
CASES = {
    # index: w_i ; partial p_i = w_i 2^-6
    "cancellation": {0: 2.0**60, 1: 3.0, 2: -2.0**60, 3: 5.0},
    "above_tie": {0: 2.0**59, 1: 2.0**6, 2: 2.0**-2},
    "tie_to_even": {0: 2.0**59, 1: 2.0**6},
    "mixed_signs": {0: -2.0**61, 1: 7.0, 2: 2.0**61, 3: -2.0**3, 5: 2.0**40, 6: -2.0**40},
}


def exact_h(ws):
    total = sum(Fraction(w) * Fraction(1, 64) for w in ws.values())
    return float(total)  # correctly rounded (Fraction -> float rounds to nearest even)


@pytest.mark.parametrize("name", sorted(CASES))
def test_first_projection_is_the_rounded_exact_sum(lib, name):
    from paper_2509_23180_gb300 import binding as B
    d = B.Domain(B.make_desc("cross", 8, 0.0, nrhs=1))
    d.set_option(B.OPT_ARNOLDI_CLUSTER, 1)  # the register-resident cluster kernel
    v0 = np.full(LEN, 2.0**-6)
    w = np.zeros(LEN)
    for i, x in CASES[name].items():
        w[i] = x
    V = torch.as_tensor(v0[None, None, :], dtype=torch.float64, device="cuda")
    wd = torch.as_tensor(w[None, :], dtype=torch.float64, device="cuda")
    h = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    d.arnoldi_mgs(V, 0, wd, h, LEN, 1)
    torch.cuda.synchronize()
    got = h.cpu().numpy()[0, 0]
    want = exact_h(CASES[name])
    assert got == want, (name, got.hex(), want.hex())
    d.close()


def test_the_norm_closing_the_step_is_exact_too(lib):
    """After the projection, ||w - h v_0|| of a w that is already orthogonal to v_0
    (h = 0 exactly) is the square root of an exact sum of squares."""
    from paper_2509_23180_gb300 import binding as B
    d = B.Domain(B.make_desc("cross", 8, 0.0, nrhs=1))
    d.set_option(B.OPT_ARNOLDI_CLUSTER, 1)
    v0 = np.full(LEN, 2.0**-6)
    w = np.zeros(LEN)
    w[0], w[1], w[2], w[3] = 2.0**30, -2.0**30, 1.0, -1.0  # (w, v_0) = 0
    V = torch.as_tensor(v0[None, None, :], dtype=torch.float64, device="cuda")
    wd = torch.as_tensor(w[None, :], dtype=torch.float64, device="cuda")
    h = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    d.arnoldi_mgs(V, 0, wd, h, LEN, 1)
    torch.cuda.synchronize()
    hh = h.cpu().numpy()[0]
    assert hh[0] == 0.0
    want = float(np.sqrt(float(sum(Fraction(x) ** 2 for x in (2.0**30, -2.0**30, 1.0, -1.0)))))
    assert hh[1] == want
    d.close()
