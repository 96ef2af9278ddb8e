"""Pins for Algorithm 1 (ADM for the l1 regression of Eq. l1g).

The exact answer of min_z ||x - A z||_1 is fixed by linear programming, not by
the ADM: brute-force vertex enumeration (tiny cases), SciPy's HiGHS LP, and a
KKT/subgradient certificate.  Special cases: with no corruption the first
iteration returns the least-squares fit z = A^T x and stops; a column of zeros
needs no iteration; exact recovery of z0 when the corruption is sparse.
"""
import numpy as np
import pytest

from oracle import l1filter, lp

scipy = pytest.importorskip("scipy")


def _basis(rng, p, r):
    A, _ = np.linalg.qr(rng.standard_normal((p, r)))
    return A


def _problem(rng, p, r, N, dens, mag=50.0, zscale=10.0):
    A = _basis(rng, p, r)
    Z0 = rng.standard_normal((r, N)) * zscale
    S = (rng.random((p, N)) < dens) * rng.uniform(-mag, mag, (p, N))
    return A, Z0, A @ Z0 + S


def test_adm_matches_bruteforce_vertex_enumeration():
    # seeds have at least 10r rows (Section 3.1), so p >= 10 r here
    rng = np.random.default_rng(10)
    for (p, r) in [(20, 2), (24, 2), (30, 3)]:
        A, Z0, X = _problem(rng, p, r, 12, 0.15)
        res = l1filter.adm_l1(X, A)
        assert res.converged.all()
        for j in range(X.shape[1]):
            zb, vb = lp.l1_regression_bruteforce(X[:, j], A)
            va = np.abs(X[:, j] - A @ res.Z[:, j]).sum()
            assert va <= vb + 1e-7 * max(1.0, vb), (p, r, j, va, vb)


def test_adm_matches_lp_optimum():
    rng = np.random.default_rng(11)
    for (p, r, dens) in [(50, 5, 0.1), (50, 5, 0.2), (200, 20, 0.1),
                         (200, 20, 0.3)]:
        A, Z0, X = _problem(rng, p, r, 40, dens)
        res = l1filter.adm_l1(X, A)
        for j in range(X.shape[1]):
            zl, vl = lp.l1_regression_lp(X[:, j], A)
            va = np.abs(X[:, j] - A @ res.Z[:, j]).sum()
            assert va <= vl * (1 + 1e-8) + 1e-9, (p, r, dens, j, va, vl)
            assert np.linalg.norm(res.Z[:, j] - zl) <= \
                1e-7 * max(1.0, np.linalg.norm(zl))


def test_adm_kkt_certificate():
    rng = np.random.default_rng(12)
    A, Z0, X = _problem(rng, 60, 4, 20, 0.15)
    res = l1filter.adm_l1(X, A)
    for j in range(X.shape[1]):
        gmax, eqres = lp.kkt_certificate(X[:, j], A, res.Z[:, j])
        assert gmax <= 1 + 1e-6 and eqres <= 1e-6


def test_adm_exact_recovery_sparse_corruption():
    # Section 3.4: sparse enough S^c is recovered exactly
    rng = np.random.default_rng(13)
    A, Z0, X = _problem(rng, 200, 20, 64, 0.1, mag=100.0)
    res = l1filter.adm_l1(X, A)
    err = np.linalg.norm(res.Z - Z0) / np.linalg.norm(Z0)
    assert err < 1e-9


def test_adm_no_corruption_is_least_squares_in_one_step():
    rng = np.random.default_rng(14)
    A = _basis(rng, 40, 6)
    X = A @ rng.standard_normal((6, 7))
    res = l1filter.adm_l1(X, A)
    np.testing.assert_allclose(res.Z, A.T @ X, rtol=0, atol=1e-12)
    assert (res.iters == 1).all()
    assert np.abs(res.E).max() == 0.0


def test_adm_zero_column_takes_no_iteration():
    rng = np.random.default_rng(15)
    A = _basis(rng, 20, 3)
    X = np.zeros((20, 3))
    X[:, 1] = A @ np.array([1.0, -2.0, 0.5])
    res = l1filter.adm_l1(X, A)
    assert res.iters[0] == 0 and res.iters[2] == 0
    assert np.all(res.Z[:, 0] == 0) and np.all(res.Z[:, 2] == 0)
    assert res.converged.all()


def test_adm_single_outlier_by_hand():
    # rank-1 basis, one corrupted entry: the exact solution is the clean fit
    p = 9
    a = np.ones(p) / 3.0  # unit norm
    A = a[:, None]
    x = 2.0 * a
    x[4] += 100.0
    res = l1filter.adm_l1(x, A)
    assert abs(res.Z[0, 0] - 2.0) < 1e-9
    e = x - 2.0 * a
    np.testing.assert_allclose(res.E[:, 0], e, atol=1e-8)


def test_adm_planted_transpose_mistake_is_caught():
    # A copy of step 2 with A in place of A^T (a plausible slip) gives the
    # wrong answer, which the LP pin exposes.
    rng = np.random.default_rng(16)
    A, Z0, X = _problem(rng, 6, 6, 1, 0.0)
    A = A + 0.1 * rng.standard_normal(A.shape)  # non-symmetric square basis
    A, _ = np.linalg.qr(A)
    x = X[:, 0]
    z_bad = A @ x  # the slip: A instead of A^T
    zl, vl = lp.l1_regression_lp(x, A)
    assert np.abs(x - A @ z_bad).sum() > vl + 1e-6


def test_lp_and_bruteforce_agree():
    # the two exact solvers pin each other (independent methods)
    rng = np.random.default_rng(17)
    for (p, r) in [(12, 2), (16, 3)]:
        A, Z0, X = _problem(rng, p, r, 6, 0.3)
        for j in range(X.shape[1]):
            zb, vb = lp.l1_regression_bruteforce(X[:, j], A)
            zl, vl = lp.l1_regression_lp(X[:, j], A)
            assert abs(vb - vl) <= 1e-8 * max(1.0, vb)


def test_adm_nonunique_minimiser_reaches_the_optimal_objective():
    # degenerate l1 regressions whose minimisers form a segment: z is not
    # unique, so the ADM's answer is checked by its objective (against the
    # closed form and the LP) and by membership of the optimal set
    a1 = np.array([1, 1, 1, 1, 0, 0, 0, 0]) / 2.0
    a2 = np.array([0, 0, 0, 0, 1, 1, 1, 1]) / 2.0
    A = np.stack([a1, a2], axis=1)                   # orthonormal columns
    x = np.array([0.0, 0.0, 1.0, 1.0, 0.0, 1.0, 2.0, 3.0])
    # separable: sum |x_i - z1/2| over {0, 0, 1, 1} is 2 for z1/2 in [0, 1];
    # over {0, 1, 2, 3} it is 4 for z2/2 in [1, 2] (any median)
    res = l1filter.adm_l1(x[:, None], A)
    assert res.converged.all()
    z = res.Z[:, 0]
    va = np.abs(x - A @ z).sum()
    _, vl = lp.l1_regression_lp(x, A)
    assert abs(va - 6.0) <= 1e-9 * 6.0 and abs(vl - 6.0) <= 1e-9 * 6.0
    tol = 1e-8
    assert -tol <= z[0] / 2 <= 1 + tol and 1 - tol <= z[1] / 2 <= 2 + tol
    gmax, eqres = lp.kkt_certificate(x, A, z)
    assert gmax <= 1 + 1e-6 and eqres <= 1e-6
    # one column of a single basis vector: any z/2 in [0, 1] is optimal
    A1 = np.full((4, 1), 0.5)
    x1 = np.array([0.0, 0.0, 1.0, 1.0])
    r1 = l1filter.adm_l1(x1[:, None], A1)
    z1 = r1.Z[0, 0]
    assert abs(np.abs(x1 - A1[:, 0] * z1).sum() - 2.0) <= 1e-9 * 2.0
    assert -tol <= z1 / 2 <= 1 + tol
