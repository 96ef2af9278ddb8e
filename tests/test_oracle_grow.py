"""Oracle pins for the seed-size rule of Section 3.5 (target rank test).

When the seed's rank r' fails Eq. rank_test (m'/r' >= s_r, n'/r' >= s_c),
the seed grows to (s_r r') x (s_c r') and the procedure repeats, until the
test holds or the seed would exceed half of a side (Eq. rank_test1).
Seeds here are prefixes of fixed row / column orders.
"""
import numpy as np

from oracle import l1filter
from paper_1108_5359_gb300 import synth


def _instance(seed, m=600, n=560, r=5, dens=0.12):
    M, L0, S0 = synth.lowrank_plus_sparse(m, n, r, dens, -50, 50,
                                          seed=(seed, 77))
    rng = np.random.default_rng(seed)
    return M, L0, S0, rng.permutation(m), rng.permutation(n)


def _first_seed(M, ro, co, mp, np_, r):
    return l1filter.l1_filter_pcp(M, np.sort(ro[:mp]), np.sort(co[:np_]), r=r)


def test_failed_seed_grows_by_the_rule_and_recovers():
    M, L0, S0, ro, co = _instance(0)
    first = _first_seed(M, ro, co, 50, 50, 5)
    assert not first.rank_ok and first.rank_raw > 5     # 50 x 50 too small
    res, sizes = l1filter.l1_filter_pcp_grow(M, ro, co, r=5)
    assert sizes[0] == (50, 50)
    assert sizes[1] == (10 * first.rank_raw, 10 * first.rank_raw)
    assert res.rank_ok and res.rank == 5
    assert np.linalg.norm(res.L - L0) / np.linalg.norm(L0) < 1e-6
    assert np.linalg.norm(res.S - S0) / np.linalg.norm(S0) < 1e-6


def test_passing_seed_is_kept():
    M, L0, S0, ro, co = _instance(3)
    res, sizes = l1filter.l1_filter_pcp_grow(M, ro, co, r=5)
    assert sizes == [(50, 50)]
    ref = _first_seed(M, ro, co, 50, 50, 5)
    np.testing.assert_array_equal(res.L, ref.L)


def test_growth_stops_at_half_of_a_side():
    # heavy corruption on a small matrix: every seed the rule asks for would
    # exceed half of a side, so the method gives up (Eq. rank_test1)
    M, L0, S0, ro, co = _instance(1, m=130, n=120, r=5, dens=0.35)
    res, sizes = l1filter.l1_filter_pcp_grow(M, ro, co, r=5)
    assert all(mp <= 65 and np_ <= 60 for mp, np_ in sizes)
    assert not res.rank_ok
    assert sizes == sorted(sizes)        # never shrinks
