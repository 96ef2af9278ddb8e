"""Pins for the shrinkage operator and singular value thresholding.

Shrinkage S_eta(x) = sgn(x) max(|x| - eta, 0) and SVT (Eq. Proxy / Eq. SVT,
Section 2).  Checked against closed forms and the optimality conditions of the
two proximal problems, never against the oracle's own formula.
"""
import numpy as np

from oracle import pcp


def test_soft_threshold_closed_form_points():
    # S_eta is the prox of eta*|x|: values fixed by hand
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.5])
    got = pcp.soft_threshold(x, 1.0)
    np.testing.assert_array_equal(got, [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.5])


def test_soft_threshold_is_prox_of_l1():
    # argmin_y eta|y| + (y - x)^2 / 2, found by dense search, equals S_eta(x)
    rng = np.random.default_rng(0)
    grid = np.linspace(-10, 10, 200001)
    for _ in range(20):
        x = rng.uniform(-8, 8)
        eta = rng.uniform(0.01, 3)
        obj = eta * np.abs(grid) + 0.5 * (grid - x) ** 2
        y = grid[np.argmin(obj)]
        assert abs(pcp.soft_threshold(x, eta) - y) <= 1e-4


def test_svt_diagonal_reduces_to_shrinkage():
    s = np.array([5.0, 3.0, 1.0, 0.2])
    W = np.diag(s)
    A, U, sp, Vt = pcp.svt(W, 0.5)
    np.testing.assert_allclose(A, np.diag([4.5, 2.5, 0.5, 0.0]), atol=1e-14)
    np.testing.assert_allclose(sp, [4.5, 2.5, 0.5])


def test_svt_optimality_condition():
    # W - A must lie in eta * subdifferential of the nuclear norm at A:
    # W - A = eta (U V^T + R), U^T R = 0, R V = 0, ||R||_2 <= 1.
    rng = np.random.default_rng(1)
    W = rng.standard_normal((30, 20)) @ np.diag(np.linspace(5, 0.1, 20))
    eta = 1.3
    A, U, sp, Vt = pcp.svt(W, eta)
    G = (W - A) / eta
    R = G - U @ Vt
    assert np.abs(U.T @ R).max() < 1e-12
    assert np.abs(R @ Vt.T).max() < 1e-12
    assert np.linalg.norm(R, 2) <= 1 + 1e-12


def test_svt_objective_beats_perturbations():
    rng = np.random.default_rng(2)
    W = rng.standard_normal((12, 9))
    eta = 0.7

    def f(A):
        return eta * np.linalg.svd(A, compute_uv=False).sum() + \
            0.5 * np.linalg.norm(A - W) ** 2

    A, *_ = pcp.svt(W, eta)
    base = f(A)
    for _ in range(200):
        assert f(A + 1e-3 * rng.standard_normal(A.shape)) >= base - 1e-12


def test_svt_planted_wrong_sign_is_caught():
    # A mistake planted in a copy of the prox (adding eta instead of
    # subtracting) must violate the optimality condition above.
    rng = np.random.default_rng(3)
    W = rng.standard_normal((10, 8))
    eta = 0.5
    U, s, Vt = np.linalg.svd(W, full_matrices=False)
    A_bad = (U * (s + eta)) @ Vt
    G = (W - A_bad) / eta
    R = G - U @ Vt
    assert np.linalg.norm(R, 2) > 1 + 1e-6 or \
        np.abs(U.T @ R).max() > 1e-6
