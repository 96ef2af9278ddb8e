"""The plain-FP32 variant of the oracle (the same steps with dtype=float32).

Pinned by what the mathematics fixes, not by the FP64 oracle's output:
exact recovery of L0 and S0 (Section 4.1.1's generator; the method
recovers them exactly in exact arithmetic), here to FP32 accuracy, with the
same Eq. rank_test outcome, every array in FP32, and the seed ALM reaching
its 1e-7 stop rule.
"""
import numpy as np

from oracle import l1filter
from paper_1108_5359_gb300 import synth


def _relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) /
                 np.linalg.norm(b))


def test_fp32_variant_recovers_l0_and_s0():
    P = synth.make_config("c1_500_r5", seed=4, m=1000, n=900, r=8)
    res = l1filter.l1_filter_pcp(P.M.astype(np.float32), P.rows, P.cols,
                                 r=P.r, adm_kw=dict(eps=1e-6),
                                 dtype=np.float32)
    assert res.L.dtype == np.float32 and res.S.dtype == np.float32
    assert res.Lu.dtype == np.float32 and res.Qt.dtype == np.float32
    assert res.rank_ok and res.rank == P.r
    assert res.seed_residual <= 1e-7
    assert _relerr(res.L, P.L0) < 2e-5
    assert _relerr(res.S, P.S0) < 2e-5


def test_fp32_variant_single_regression_brute_force():
    # one l1 regression with a unique minimiser: A = e_1 (p x 1), x with
    # outliers on a minority of entries; the minimiser of ||x - a z||_1 is
    # the median of x over the support of a, i.e. x_0 here
    p = 9
    A = np.zeros((p, 1), np.float32)
    A[0, 0] = 1.0
    x = np.linspace(1.0, 2.0, p).astype(np.float32)
    res = l1filter.adm_l1(x[:, None], A, eps=1e-6, dtype=np.float32)
    assert res.Z.dtype == np.float32
    assert abs(float(res.Z[0, 0]) - float(x[0])) < 1e-5
