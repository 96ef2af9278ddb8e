"""The oracle on the second workload shapes of Section 4.1.2.

The paper reports that l1 filtering keeps recovering L0 when the sparse part
is scaled up (M = L0 + sigma S0, sigma from 1 to 10, m = 1000, r = 0.01 m,
support ratio 0.01), measured by RelErr, MaxDif = max |L* - L0| and AveDif =
sum |L* - L0| / m^2; and that it recovers the deterministic rank-2
checkerboard under 10% impulsive noise.  These pin the oracle end to end on
inputs with known answers.  The bounds follow from the inputs: M is rounded
to FP32 (the GPU path's input), so the recovered L0 can be exact only to the
FP32 rounding of M, and the ADM stop rule is relative to the data, whose
scale grows with sigma.
"""
import numpy as np
import pytest

from oracle import l1filter
from paper_1108_5359_gb300 import synth


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("sigma", [1.0, 3.0, 10.0])
def test_sparse_magnitude_sweep_recovers_L0(sigma):
    P = synth.sparse_magnitude(sigma, m=1000, seed=1)
    assert P.r == 10 and np.count_nonzero(P.S0) == 10_000
    assert np.abs(P.S0).max() <= 500 * sigma
    M = P.M.astype(np.float32).astype(np.float64)
    ref = l1filter.l1_filter_pcp(M, P.rows, P.cols, r=P.r)
    assert ref.rank == P.r
    assert _relerr(ref.L, P.L0) < 1e-5
    assert _relerr(ref.S, P.S0) < 1e-6
    max_dif = np.abs(ref.L - P.L0).max()
    ave_dif = np.abs(ref.L - P.L0).sum() / P.m ** 2
    # the FP32 rounding of M alone moves entries by up to |M| 2^-24
    assert max_dif < 1e-3 and ave_dif < 1e-5
    # the support of S0 is found exactly
    found = np.abs(ref.S) > 1e-2
    np.testing.assert_array_equal(found, P.S0 != 0)


@pytest.mark.parametrize("m", [1000, 1500])
def test_checkerboard_is_recovered(m):
    P = synth.checkerboard(m, seed=0)
    assert np.linalg.matrix_rank(P.L0) == 2
    # impulsive noise: each corrupted entry takes the opposite colour
    flipped = P.S0 != 0
    assert abs(flipped.mean() - 0.10) < 1e-3
    np.testing.assert_array_equal(P.M[flipped], 1.0 - P.L0[flipped])
    ref = l1filter.l1_filter_pcp(P.M, P.rows, P.cols, r=2)
    assert ref.rank == 2
    assert _relerr(ref.L, P.L0) < 1e-6
    assert _relerr(ref.S, P.S0) < 1e-6
    # the recovered image rounds back to the checkerboard
    np.testing.assert_array_equal(np.rint(ref.L), P.L0)


def test_checkerboard_small_seed_does_not_recover():
    # a 20 x 20 seed (10 r) at 10% corruption: the seed PCP itself misses
    # L0 on the seed, and the filters carry the error to the whole matrix
    P = synth.checkerboard(1000, seed=0, seed_size=20)
    ref = l1filter.l1_filter_pcp(P.M, P.rows, P.cols, r=2)
    blk = np.ix_(P.rows, P.cols)
    assert _relerr(ref.L[blk], P.L0[blk]) > 1e-2
    assert _relerr(ref.L, P.L0) > 1e-2
