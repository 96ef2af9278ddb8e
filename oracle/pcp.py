"""Soft shrinkage, singular value thresholding and inexact-ALM PCP (FP64;
the same steps in FP32 through ``dtype`` for the plain-FP32 variant).

Test infrastructure only (see ``oracle/__init__``).

* ``soft_threshold`` -- the shrinkage operator S_eta(x) = sgn(x) max(|x| - eta, 0)
  (Section 2, defined beside Eq. SVT).
* ``svt``            -- the closed-form minimiser of
  eta ||A||_* + 1/2 ||A - W||_F^2, i.e. U S_eta(Sigma) V^T (Eq. Proxy, Eq. SVT).
* ``inexact_alm_pcp`` -- ADM (inexact augmented Lagrange multipliers) for
  min ||L||_* + lam ||S||_1 s.t. D = L + S (Eq. PCP; Eq. SPCP for the seed).
  The paper solves the seed "e.g. using ADM" of its reference
  [lin2009augmented] and omits the pseudo code (Section 3.2 footnote), so the
  steps below are that method written out: SVT on L, shrink on S, dual ascent
  on Y, geometric growth of the penalty mu.  The constants (Y0, mu0, rho,
  mu_max) are this oracle's reading and are listed in the design notes.
  Stopping rule ||D - L - S||_F / ||D||_F <= tol with tol = 1e-7, the rule
  Section 4.1.1 uses for every method.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["soft_threshold", "svt", "inexact_alm_pcp", "PCPResult"]


def soft_threshold(x, eta, dtype=np.float64):
    """S_eta(x) = sgn(x) * max(|x| - eta, 0), elementwise (Section 2).

    ``eta`` may be a scalar or broadcast against ``x``; sgn(0) = 0 so
    S_eta(0) = 0.  ``dtype``: the arithmetic (FP64; FP32 for the plain-FP32
    variant).
    """
    x = np.asarray(x, dtype=dtype)
    return np.sign(x) * np.maximum(np.abs(x) - eta, 0.0)


def svt(W, eta, dtype=np.float64):
    """Singular value thresholding (Eq. SVT).

    Returns (A, U_+, s_+, Vt_+) with A = U S_eta(Sigma) V^T computed from a full
    LAPACK SVD of W, and the skinny factors of A restricted to the singular
    values that survive (sigma_i > eta), s_+ = sigma_i - eta.
    """
    U, s, Vt = np.linalg.svd(np.asarray(W, dtype=dtype),
                             full_matrices=False)
    keep = s > eta
    s_shr = s[keep] - eta
    Uk = U[:, keep]
    Vtk = Vt[keep, :]
    A = (Uk * s_shr) @ Vtk
    return A, Uk, s_shr, Vtk


@dataclasses.dataclass
class PCPResult:
    L: np.ndarray
    S: np.ndarray
    U: np.ndarray       # skinny SVD of L from the last SVT step
    sigma: np.ndarray
    V: np.ndarray       # n x rank (V, not V^T)
    iters: int
    residual: float     # ||D - L - S||_F / ||D||_F at exit
    converged: bool


def inexact_alm_pcp(D, lam, tol=1e-7, rho=1.5, mu_scale=1.25,
                    mu_max_ratio=1e7, max_iter=1000, dtype=np.float64):
    """Solve min ||L||_* + lam ||S||_1 s.t. D = L + S by inexact ALM.

    Steps per iteration k (the ADM of the cited solver, in the paper's
    notation: SVT for the nuclear-norm block, shrinkage for the l1 block):

      L_{k+1} = SVT_{1/mu_k}(D - S_k + Y_k / mu_k)
      S_{k+1} = S_{lam/mu_k}(D - L_{k+1} + Y_k / mu_k)
      Y_{k+1} = Y_k + mu_k (D - L_{k+1} - S_{k+1})
      mu_{k+1} = min(rho mu_k, mu_max)

    with S_0 = 0, Y_0 = D / max(||D||_2, ||D||_inf / lam),
    mu_0 = mu_scale / ||D||_2, mu_max = mu_max_ratio * mu_0, and stop when
    ||D - L - S||_F / ||D||_F <= tol.

    ``dtype`` sets the arithmetic: FP64 (the oracle), or FP32 for the
    plain-FP32 variant (same steps and constants).
    """
    D = np.asarray(D, dtype=dtype)
    normF = np.linalg.norm(D, "fro")
    if normF == 0.0:
        z = np.zeros_like(D)
        return PCPResult(z, z.copy(), np.zeros((D.shape[0], 0), dtype),
                         np.zeros(0, dtype), np.zeros((D.shape[1], 0), dtype),
                         0, 0.0, True)
    norm2 = np.linalg.norm(D, 2)
    norminf = np.abs(D).max() / lam
    Y = D / max(norm2, norminf)
    mu = mu_scale / norm2
    mu_max = mu * mu_max_ratio
    S = np.zeros_like(D)
    L = np.zeros_like(D)
    U = np.zeros((D.shape[0], 0), dtype)
    s = np.zeros(0, dtype)
    Vt = np.zeros((0, D.shape[1]), dtype)
    it = 0
    res = 1.0
    converged = False
    while it < max_iter:
        it += 1
        L, U, s, Vt = svt(D - S + Y / mu, 1.0 / mu, dtype)
        S = soft_threshold(D - L + Y / mu, lam / mu, dtype)
        Z = D - L - S
        Y = Y + mu * Z
        mu = min(rho * mu, mu_max)
        res = np.linalg.norm(Z, "fro") / normF
        if res <= tol:
            converged = True
            break
    return PCPResult(L=L, S=S, U=U, sigma=s, V=Vt.T, iters=it, residual=res,
                     converged=converged)
