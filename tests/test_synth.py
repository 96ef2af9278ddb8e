"""Seeded input generators: shapes, ranges and structure of each workload."""
import numpy as np

from paper_1108_5359_gb300 import synth


def test_uneven_instances_ranges_and_seed_sets():
    Ps = synth.uneven_instances(count=12, seed=4, m_range=(300, 900),
                                n_range=(200, 700), r_max=30)
    assert len(Ps) == 12
    for P in Ps:
        assert 300 <= P.m <= 900 and 200 <= P.n <= 700
        assert 3 <= P.r <= max(3, min(30, min(P.m, P.n) // 20))
        for idx, size in ((P.rows, P.m), (P.cols, P.n)):
            assert idx.size == 10 * P.r
            assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < size
        assert np.allclose(P.M, P.L0 + P.S0)
        assert np.linalg.matrix_rank(P.L0) == P.r
    # same seed, same instances
    Q = synth.uneven_instances(count=12, seed=4, m_range=(300, 900),
                               n_range=(200, 700), r_max=30)
    assert all(np.array_equal(a.M, b.M) for a, b in zip(Ps, Q))


def test_video_like_shape_and_foreground():
    P = synth.video_like(40, height=24, width=32, r=2, seed=1)
    assert P.M.shape == (24 * 32, 40)
    assert np.allclose(P.M, P.L0 + P.S0)
    frac = np.count_nonzero(P.S0) / P.S0.size
    assert 0.02 <= frac <= 0.2
    nz = P.S0[P.S0 != 0]
    assert nz.min() >= 0.2 - 1e-12 and nz.max() <= 1.0 + 1e-12


def test_sparse_magnitude_scales_one_sparse_part():
    # the sweep multiplies the same S0 by sigma (M = L0 + sigma S0)
    a = synth.sparse_magnitude(1.0, m=300, seed=5)
    b = synth.sparse_magnitude(7.5, m=300, seed=5)
    np.testing.assert_array_equal(a.L0, b.L0)
    np.testing.assert_array_equal(b.S0, 7.5 * a.S0)
    np.testing.assert_array_equal(b.M, b.L0 + b.S0)
    assert a.r == 3 and np.count_nonzero(a.S0) == 900
    assert np.abs(a.S0).max() <= 500.0
    np.testing.assert_array_equal(a.rows, b.rows)
    assert len(a.rows) == len(a.cols) == 30


def test_checkerboard_structure():
    P = synth.checkerboard(64, square=8, seed=2)
    i = np.arange(64) // 8 % 2
    np.testing.assert_array_equal(P.L0, (i[:, None] ^ i[None, :]))
    assert set(np.unique(P.M)) <= {0.0, 1.0}
    assert np.count_nonzero(P.S0) == round(0.10 * 64 * 64)
    assert len(P.rows) == len(P.cols) == 60
    assert np.all(np.diff(P.rows) > 0)
