"""Algorithm 1 (ADM for l1 regression) and Algorithm 2 (l1 filtering), FP64
(the same steps in FP32 through ``dtype``: the plain-FP32 variant timed
beside the oracle as a CPU baseline).

Test infrastructure only (see ``oracle/__init__``).

Algorithm 1 solves Eq. l1g,  min ||E||_1  s.t.  X = A Z + E  with A^T A = I,
by alternating minimisation of its augmented Lagrangian:

  Step 1  E_{k+1} = S_{1/beta_k}(X - A Z_k + Y_k / beta_k)
  Step 2  Z_{k+1} = A^T (X - E_{k+1} + Y_k / beta_k)
  Step 3  Y_{k+1} = Y_k + beta_k (X - A Z_{k+1} - E_{k+1}),
          beta_{k+1} = min(rho beta_k, beta_bar)

while ||X - A Z_k - E_k||_inf / ||X||_inf >= eps, from E_0 = Z_0 = Y_0 = 0.

The columns of Eq. l1g are independent problems (Section 3.2: the columns of
L^c and rows of L^r are computed independently).  Each column runs its own
instance of Algorithm 1: its own beta (beta_0 = beta0_scale / ||x||_inf,
beta_bar = beta_bar_ratio * beta_0) and its own stop test.  This per-column
reading, and the constants, are this oracle's; the paper fixes only
eps > 0, rho > 1 and beta_bar >> beta_0 > 0.  A column with ||x||_inf = 0 has
the solution z = 0, e = 0 and takes no iteration.

Algorithm 2: sample the seed (step 1; here the index sets are inputs), solve
the seed PCP (step 2, Eq. SPCP with lambda~ = 1/sqrt(max(m', n'))), filter the
columns of M^c against U^s (step 3, Eq. l1c') and the rows of M^r against V^s
(step 4, Eq. l1r'), represent the complement by
L~^s = P~^T (Sigma^s)^{-1} Q~ (step 5, Eq. l1s'), and output L and S = M - L.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .pcp import inexact_alm_pcp, soft_threshold

__all__ = ["adm_l1", "ADMResult", "l1_filter_pcp", "L1FilterResult",
           "nystrom_factors", "numerical_rank", "rank_test"]

# Defaults of this oracle's reading of Algorithm 1 (FP64).
ADM_EPS = 1e-10
ADM_RHO = 1.5
ADM_BETA0_SCALE = 1.0
ADM_BETA_BAR_RATIO = 1e10
ADM_MAX_ITER = 1000


@dataclasses.dataclass
class ADMResult:
    Z: np.ndarray        # r x N
    E: np.ndarray        # p x N
    iters: np.ndarray    # per column
    converged: np.ndarray


def adm_l1(X, A, eps=ADM_EPS, rho=ADM_RHO, beta0_scale=ADM_BETA0_SCALE,
           beta_bar_ratio=ADM_BETA_BAR_RATIO, max_iter=ADM_MAX_ITER,
           dtype=np.float64):
    """Algorithm 1 on every column of X (p x N) with basis A (p x r).

    A must have orthonormal columns (A^T A = I), which is what lets step 2 be
    a plain product with A^T.  ``dtype``: FP64 (the oracle) or FP32 (the
    plain-FP32 variant, which needs an eps above FP32 resolution).
    """
    X = np.asarray(X, dtype=dtype)
    A = np.asarray(A, dtype=dtype)
    if X.ndim == 1:
        X = X[:, None]
    p, N = X.shape
    r = A.shape[1]
    xinf = np.abs(X).max(axis=0) if p > 0 else np.zeros(N, dtype)
    Z = np.zeros((r, N), dtype)
    E = np.zeros((p, N), dtype)
    Y = np.zeros((p, N), dtype)
    AZ = np.zeros((p, N), dtype)
    active = xinf > 0
    safe = np.where(active, xinf, 1.0)
    beta = beta0_scale / safe
    beta_bar = beta_bar_ratio * beta
    iters = np.zeros(N, dtype=np.int64)
    converged = ~active.copy()
    for _ in range(max_iter + 1):
        # loop condition: ||X - A Z_k - E_k||_inf / ||X||_inf >= eps
        rel = (np.abs(X - AZ - E).max(axis=0) / safe if p > 0
               else np.zeros(N, dtype))
        done = active & (rel < eps)
        converged |= done
        active &= ~done
        if not active.any():
            break
        if iters.max(initial=0) >= max_iter:
            break
        c = active
        Xc, Yc, b = X[:, c], Y[:, c], beta[c]
        # Step 1
        Ec = soft_threshold(Xc - AZ[:, c] + Yc / b, 1.0 / b, dtype)
        # Step 2
        Zc = A.T @ (Xc - Ec + Yc / b)
        # Step 3
        AZc = A @ Zc
        Yc = Yc + b * (Xc - AZc - Ec)
        E[:, c], Z[:, c], AZ[:, c], Y[:, c] = Ec, Zc, AZc, Yc
        beta[c] = np.minimum(rho * b, beta_bar[c])
        iters[c] += 1
    return ADMResult(Z=Z, E=E, iters=iters, converged=converged)


def numerical_rank(sigma, rel_cut=1e-6):
    """Count singular values above rel_cut * sigma_max."""
    sigma = np.asarray(sigma)
    if sigma.size == 0 or sigma.max() <= 0:
        return 0
    return int(np.sum(sigma > rel_cut * sigma.max()))


def rank_test(mp, np_, r_est, s_r=10.0, s_c=10.0):
    """Eq. rank_test: accept the seed if m'/r' >= s_r and n'/r' >= s_c."""
    if r_est <= 0:
        return False
    return (mp / r_est >= s_r) and (np_ / r_est >= s_c)


def nystrom_factors(m, n, rows, cols, U, sigma, V, Pt, Qt, dtype=np.float64):
    """Factors of L = Lu diag(W) Lv^T (Eq. l1s', Algorithm 2 step 5).

    Lu[I_s] = U^s Sigma^s, Lu[~I_s] = P~^T; Lv[J_s] = V^s Sigma^s,
    Lv[~J_s] = Q~^T; W = (Sigma^s)^{-1}.  Then the four blocks of L are
    U Sigma V^T, U Q~, P~^T V^T and P~^T Sigma^{-1} Q~.
    """
    r = sigma.size
    rbar = np.setdiff1d(np.arange(m), rows)
    cbar = np.setdiff1d(np.arange(n), cols)
    Lu = np.zeros((m, r), dtype)
    Lv = np.zeros((n, r), dtype)
    Lu[rows] = U * sigma
    Lu[rbar] = Pt.T
    Lv[cols] = V * sigma
    Lv[cbar] = Qt.T
    W = 1.0 / sigma
    return Lu, Lv, W


@dataclasses.dataclass
class L1FilterResult:
    L: np.ndarray
    S: np.ndarray
    Lu: np.ndarray
    Lv: np.ndarray
    W: np.ndarray
    U: np.ndarray
    sigma: np.ndarray
    V: np.ndarray
    rank: int
    rank_ok: bool
    rank_raw: int
    seed_iters: int
    seed_residual: float
    col_iters: np.ndarray
    row_iters: np.ndarray
    Qt: np.ndarray
    Pt: np.ndarray


def l1_filter_pcp(M, rows, cols, r=None, seed_tol=1e-7, lam_seed=None,
                  s_r=10.0, s_c=10.0, rank_cut=1e-6, adm_kw=None,
                  seed_kw=None, form_L=True, dtype=np.float64):
    """Algorithm 2 on M (m x n) with seed rows I_s = rows, columns J_s = cols.

    ``r`` caps the rank kept from the seed (the target rank); None keeps the
    numerical rank of L^s: singular values above rank_cut times the largest.
    The seed PCP stops at a relative residual of 1e-7, so L^s is resolved
    only to about 1e-7 of its norm; components below 1e-6 of the largest are
    treated as zero (with a 1e-10 cut, two equally converged ALM iterates
    of a borderline seed can disagree on the rank).

    ``dtype``: FP64 (the oracle) or FP32 (the plain-FP32 variant: the same
    steps in FP32 arithmetic; pass adm_kw eps >= 1e-6, which FP32 resolves).
    """
    M = np.asarray(M, dtype=dtype)
    m, n = M.shape
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    mp, np_ = rows.size, cols.size
    adm_kw = dict(adm_kw or {})
    seed_kw = dict(seed_kw or {})
    # step 2: seed PCP (Eq. SPCP)
    Ms = M[np.ix_(rows, cols)]
    if lam_seed is None:
        lam_seed = 1.0 / math.sqrt(max(mp, np_))
    seed = inexact_alm_pcp(Ms, lam_seed, tol=seed_tol, dtype=dtype, **seed_kw)
    rk_raw = numerical_rank(seed.sigma, rank_cut)
    rk = rk_raw if r is None else min(rk_raw, int(r))
    order = np.argsort(-seed.sigma)[:rk]
    U = seed.U[:, order]
    sigma = seed.sigma[order]
    V = seed.V[:, order]
    # Eq. rank_test on the seed's own numerical rank (before the cap at r)
    ok = rank_test(mp, np_, rk_raw, s_r, s_c)
    rbar = np.setdiff1d(np.arange(m), rows)
    cbar = np.setdiff1d(np.arange(n), cols)
    # step 3: column filtering, M^c = U^s Q~ + S^c (Eq. l1c')
    col = adm_l1(M[np.ix_(rows, cbar)], U, dtype=dtype, **adm_kw)
    # step 4: row filtering, (M^r)^T = V^s P~ + (S^r)^T (Eq. l1r')
    row = adm_l1(M[np.ix_(rbar, cols)].T, V, dtype=dtype, **adm_kw)
    # step 5: Nystrom representation (Eq. l1s')
    Lu, Lv, W = nystrom_factors(m, n, rows, cols, U, sigma, V, row.Z, col.Z,
                                dtype)
    if form_L:
        L = (Lu * W) @ Lv.T
        S = M - L
    else:
        L = S = None
    return L1FilterResult(L=L, S=S, Lu=Lu, Lv=Lv, W=W, U=U, sigma=sigma, V=V,
                          rank=rk, rank_ok=ok, rank_raw=rk_raw,
                          seed_iters=seed.iters,
                          seed_residual=seed.residual, col_iters=col.iters,
                          row_iters=row.iters, Qt=col.Z, Pt=row.Z)


def l1_filter_pcp_grow(M, row_order, col_order, r, s_r=10.0, s_c=10.0,
                       max_frac=0.5, **kw):
    """Algorithm 2 with the seed-size rule of Section 3.5.

    The seed is the first m' = round(s_r r) entries of ``row_order`` and the
    first n' = round(s_c r) of ``col_order`` (each sorted).  If the seed's
    rank r' fails Eq. rank_test, the seed grows to (s_r r') x (s_c r')
    (prefixes of the same orders) and the procedure repeats, until the test
    holds or the next seed would exceed max_frac of a side (Eq. rank_test1),
    where the method gives up.  The target rank r only sizes the first seed
    and caps the rank kept.

    Returns (result, sizes): the result of the last seed tried (rank_ok
    tells whether it was accepted) and the list of (m', n') tried.
    """
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    row_order = np.asarray(row_order, dtype=np.int64)
    col_order = np.asarray(col_order, dtype=np.int64)
    mp, np_ = int(round(s_r * r)), int(round(s_c * r))
    sizes = []
    res = None
    while mp <= max_frac * m and np_ <= max_frac * n:
        rows = np.sort(row_order[:mp])
        cols = np.sort(col_order[:np_])
        res = l1_filter_pcp(M, rows, cols, r=r, s_r=s_r, s_c=s_c, **kw)
        sizes.append((mp, np_))
        if res.rank_ok:
            break
        nmp = int(round(s_r * res.rank_raw))
        nnp = int(round(s_c * res.rank_raw))
        if nmp <= mp and nnp <= np_:
            break  # the rule would not grow the seed
        mp, np_ = max(nmp, mp), max(nnp, np_)
    return res, sizes
