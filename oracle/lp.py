"""Independent pins for l1 regression (Eq. l1g, one column): exact optima.

Test infrastructure only (see ``oracle/__init__``).

min_z ||x - A z||_1 is a linear program.  Its optimum is attained at a vertex,
where (for A of full column rank r in general position) r residuals vanish.
These routines do not run Algorithm 1; they give the exact answer that
Algorithm 1 must reach:

* ``l1_regression_bruteforce`` -- enumerate every r-row subset T, solve
  A_T z = x_T, keep the least ||x - A z||_1 (exact, tiny sizes only);
* ``l1_regression_lp``         -- the LP  min 1^T t  s.t. -t <= x - A z <= t,
  solved by SciPy's HiGHS;
* ``kkt_certificate``          -- optimality test: z is optimal iff some g with
  g_i = sign(res_i) where res_i != 0 and |g_i| <= 1 where res_i = 0 satisfies
  A^T g = 0 (subgradient condition of ||x - A z||_1).
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = ["l1_regression_bruteforce", "l1_regression_lp", "kkt_certificate"]


def l1_regression_bruteforce(x, A):
    """Exact l1 regression by vertex enumeration (p <= ~16, r <= 4)."""
    x = np.asarray(x, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    p, r = A.shape
    best_val = np.inf
    best_z = None
    for T in itertools.combinations(range(p), r):
        AT = A[list(T)]
        if abs(np.linalg.det(AT)) < 1e-12:
            continue
        z = np.linalg.solve(AT, x[list(T)])
        val = np.abs(x - A @ z).sum()
        if val < best_val - 1e-12:
            best_val, best_z = val, z
    return best_z, best_val


def l1_regression_lp(x, A):
    """Exact l1 regression as an LP (SciPy HiGHS); returns (z, objective)."""
    from scipy.optimize import linprog

    x = np.asarray(x, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    p, r = A.shape
    # variables [z (free, r), t (>= 0, p)]
    c = np.concatenate([np.zeros(r), np.ones(p)])
    I = np.eye(p)
    #  x - A z <= t   ->  -A z - t <= -x
    # -(x - A z) <= t ->   A z - t <=  x
    A_ub = np.block([[-A, -I], [A, -I]])
    b_ub = np.concatenate([-x, x])
    bounds = [(None, None)] * r + [(0, None)] * p
    sol = linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs")
    if not sol.success:
        raise RuntimeError(sol.message)
    z = sol.x[:r]
    return z, float(np.abs(x - A @ z).sum())


def kkt_certificate(x, A, z, delta=1e-8):
    """Return max |g_i| over the zero-residual set (<= 1 certifies optimality).

    N = {i : |res_i| > delta * max(1, ||x||_inf)} and Z its complement; find g_Z
    with A_Z^T g_Z = -A_N^T sign(res_N) of least max-norm (an LP when |Z| > r;
    least squares otherwise) and report ||g_Z||_inf and the equation residual.
    """
    x = np.asarray(x, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    res = x - A @ z
    tol = delta * max(1.0, np.abs(x).max())
    N = np.abs(res) > tol
    Zs = ~N
    rhs = -A[N].T @ np.sign(res[N])
    AZt = A[Zs].T  # r x |Z|
    if Zs.sum() == 0:
        return np.inf if np.abs(rhs).max(initial=0) > 1e-9 else 0.0, \
            float(np.abs(rhs).max(initial=0))
    from scipy.optimize import linprog

    k = AZt.shape[1]
    # minimise s s.t. AZt g = rhs, -s <= g_i <= s
    c = np.concatenate([np.zeros(k), [1.0]])
    A_eq = np.hstack([AZt, np.zeros((AZt.shape[0], 1))])
    A_ub = np.block([[np.eye(k), -np.ones((k, 1))],
                     [-np.eye(k), -np.ones((k, 1))]])
    b_ub = np.zeros(2 * k)
    sol = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=rhs,
                  bounds=[(None, None)] * k + [(0, None)], method="highs")
    if not sol.success:
        return np.inf, np.inf
    g = sol.x[:k]
    return float(np.abs(g).max()), float(np.abs(AZt @ g - rhs).max())
