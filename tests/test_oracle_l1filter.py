"""Pins for Algorithm 2 (l1 filtering) as a whole.

* exact recovery of L0 and S0 on generated inputs (Section 3.4; Table 1
  reports RelErr 1e-8 .. 1e-10 for the method);
* M = L + S, rank(L) = r (Table 1, rank column);
* the four Nystrom blocks of Eq. l1s / Eq. l1s' (seed block = U Sigma V^T,
  column block = U Q~, row block = P~^T V^T, complement
  L^r (L^s)^+ L^c computed independently with a pseudo-inverse);
* agreement with plain full-matrix PCP on tiny inputs (Table 1: both methods
  recover the same L0);
* the target-rank test of Eq. rank_test.
"""
import numpy as np
import pytest

from oracle import l1filter, pcp
from paper_1108_5359_gb300 import synth


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("seed", [3, 4])
def test_l1filter_exact_recovery_c1_shape(seed):
    P = synth.make_config("c1_500_r5", seed=seed)
    res = l1filter.l1_filter_pcp(P.M, P.rows, P.cols, r=P.r)
    assert res.rank == P.r and res.rank_ok
    assert _relerr(res.L, P.L0) < 1e-6
    assert _relerr(res.S, P.S0) < 1e-6
    # rank(L) = r
    s = np.linalg.svd(res.L, compute_uv=False)
    assert int((s > 1e-9 * s[0]).sum()) == P.r
    # M = L + S
    np.testing.assert_array_equal(res.L + res.S, res.L + (P.M - res.L))


def test_l1filter_nystrom_blocks():
    P = synth.make_config("c1_500_r5", seed=3, m=300, n=260)
    res = l1filter.l1_filter_pcp(P.M, P.rows, P.cols, r=P.r)
    I, J = P.rows, P.cols
    Ib = np.setdiff1d(np.arange(P.m), I)
    Jb = np.setdiff1d(np.arange(P.n), J)
    U, s, V = res.U, res.sigma, res.V
    Ls = (U * s) @ V.T
    np.testing.assert_allclose(res.L[np.ix_(I, J)], Ls, atol=1e-9)
    Lc = U @ res.Qt
    Lr = res.Pt.T @ V.T
    np.testing.assert_allclose(res.L[np.ix_(I, Jb)], Lc, atol=1e-9)
    np.testing.assert_allclose(res.L[np.ix_(Ib, J)], Lr, atol=1e-9)
    # Eq. l1s with an independent pseudo-inverse
    comp = Lr @ np.linalg.pinv(Ls, rcond=1e-10) @ Lc
    np.testing.assert_allclose(res.L[np.ix_(Ib, Jb)], comp,
                               atol=1e-7 * np.abs(comp).max())
    np.testing.assert_allclose(U.T @ U, np.eye(P.r), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(P.r), atol=1e-12)


def test_l1filter_agrees_with_full_pcp_tiny():
    M, L0, S0 = synth.lowrank_plus_sparse(160, 150, 3, 0.05, -30, 30, seed=9)
    rows, cols = synth.seed_indices(160, 150, 40, 40, seed=9)
    a = l1filter.l1_filter_pcp(M, rows, cols, r=3)
    b = pcp.inexact_alm_pcp(M, 1.0 / np.sqrt(160))
    assert _relerr(a.L, L0) < 1e-6
    assert _relerr(b.L, L0) < 1e-6
    assert _relerr(a.L, b.L) < 2e-6


def test_l1filter_no_corruption_reproduces_M():
    rng = np.random.default_rng(21)
    M = rng.standard_normal((120, 4)) @ rng.standard_normal((4, 110))
    rows, cols = synth.seed_indices(120, 110, 40, 40, seed=1)
    res = l1filter.l1_filter_pcp(M, rows, cols, r=4)
    assert _relerr(res.L, M) < 1e-7
    assert np.abs(res.S).max() < 1e-6 * np.abs(M).max()


def test_rank_test_equation():
    assert l1filter.rank_test(200, 200, 20)
    assert not l1filter.rank_test(200, 200, 21)
    assert not l1filter.rank_test(200, 150, 20)
    assert not l1filter.rank_test(50, 50, 0)


def test_l1filter_planted_nystrom_mistake_is_caught():
    # using Sigma instead of Sigma^{-1} in Eq. l1s' breaks exact recovery
    P = synth.make_config("c1_500_r5", seed=3, m=200, n=180)
    res = l1filter.l1_filter_pcp(P.M, P.rows, P.cols, r=P.r)
    bad = (res.Lu * res.sigma) @ res.Lv.T
    assert _relerr(bad, P.L0) > 1e-2
    good = (res.Lu * res.W) @ res.Lv.T
    assert _relerr(good, P.L0) < 1e-6
