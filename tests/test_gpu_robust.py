"""GPU parity on the second workload shapes of Section 4.1.2.

The same kernels on inputs unlike the Gaussian benchmark: the sparse part
scaled by sigma = 1..10 (m = 1000, r = 10, support ratio 0.01, values up to
5000 against low-rank entries of a few units), and the deterministic rank-2
checkerboard under 10% impulsive noise (m from 1000 to 5000, 60 x 60 seed).
The GPU's L and S match the FP64 oracle within relative Frobenius error 1e-5
and recover L0 and S0, in each precision form.
"""
import numpy as np
import pytest

from paper_1108_5359_gb300 import synth
from tests.gpuhelp import relerr
from tests.test_gpu_solve import _check, _gpu_solve

pytestmark = pytest.mark.gpu

PCP_FP32, PCP_BF16_REFINED, PCP_TF32_REFINED = 0, 1, 2


@pytest.mark.parametrize("precision", [PCP_FP32, PCP_TF32_REFINED,
                                       PCP_BF16_REFINED])
@pytest.mark.parametrize("sigma", [1.0, 3.0, 10.0])
def test_sparse_magnitude_sweep(sigma, precision):
    P = synth.sparse_magnitude(sigma, m=1000, seed=1)
    g = _gpu_solve(P, precision=precision)
    _, Lg = _check(P, g)
    assert relerr(Lg, P.L0) < 1e-5
    assert relerr(g["S"], P.S0) < 1e-6
    assert np.abs(Lg - P.L0).max() < 1e-3


@pytest.mark.parametrize("m,precision", [(1000, PCP_FP32),
                                         (2500, PCP_TF32_REFINED),
                                         (2500, PCP_BF16_REFINED),
                                         (5000, PCP_FP32)])
def test_checkerboard(m, precision):
    P = synth.checkerboard(m, seed=0)
    # the seed is 60 x 60 (30 r), not the default s_r r x s_c r
    g = _gpu_solve(P, precision=precision, seed_m=len(P.rows),
                   seed_n=len(P.cols))
    _, Lg = _check(P, g)
    assert relerr(Lg, P.L0) < 1e-5
    assert relerr(g["S"], P.S0) < 1e-5
    np.testing.assert_array_equal(np.rint(Lg), P.L0)
