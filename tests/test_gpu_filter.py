"""GPU parity of Algorithm 1 (pcp_l1_filter) against the FP64 oracle.

Each column of X is an independent l1 regression on an orthonormal basis A
(Eq. l1g).  The FP32 SIMT kernel (PCP_FP32_SIMT, eps = 3e-7; the tensor-core
kernel is covered by test_gpu_filter_tc.py) must give A z within relative
Frobenius error 1e-5 of the oracle's FP64 answer (eps = 1e-10), for column
problems (entries strided by 1) and row problems (entries strided by ldm),
ragged counts (N not a multiple of the 32 problems per CTA, p not a multiple
of 8), zero columns and uncorrupted columns.
"""
import numpy as np
import pytest

from oracle import l1filter
from tests.gpuhelp import build_and_load, idx_dev, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _problem(seed, p, r, N, dens=0.1, mag=50.0):
    rng = np.random.default_rng(seed)
    A, _ = np.linalg.qr(rng.standard_normal((p, r)))
    A = A.astype(np.float32).astype(np.float64)   # both sides see FP32 A
    Z0 = rng.standard_normal((r, N)) * 10
    S = (rng.random((p, N)) < dens) * rng.uniform(-mag, mag, (p, N))
    X = (A @ Z0 + S).astype(np.float32).astype(np.float64)
    return A, X


PCP_FP32_SIMT = 5


def _run(A, X, orientation, eps=3e-7, max_iter=500, rank=None, scale=None,
         precision=PCP_FP32_SIMT, lowp_iters=12):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    p, N = X.shape
    r = A.shape[1]
    if orientation == "col":
        M = to_dev_cm(X.astype(np.float32))            # p x N, ld p
        sp, sq = 1, M.stride(1)
    else:
        M = to_dev_cm(X.T.astype(np.float32), ld=N + 3)  # N x p, ld N+3
        sp, sq = M.stride(1), 1
    pidx = idx_dev(np.arange(p))
    qidx = idx_dev(np.arange(N))
    dA = to_dev_cm(A.astype(np.float32))
    Z = torch.full((r, N + 5), float("nan"), device="cuda").t()  # ld N+5
    iters = torch.zeros(N, dtype=torch.int32, device="cuda")
    d_rank = None if rank is None else idx_dev([rank])
    d_scale = None if scale is None else torch.as_tensor(
        np.asarray(scale, np.float32), device="cuda")
    pk.pcp_l1_filter(M, pidx, sp, qidx, sq, dA, r, Z, Z.stride(1), eps, 1.5,
                     max_iter=max_iter, d_rank=d_rank, d_scale=d_scale,
                     d_iters=iters, precision=precision,
                     lowp_iters=lowp_iters)
    torch.cuda.synchronize()
    return to_host(Z[:N, :]).T, iters.cpu().numpy()


@pytest.mark.parametrize("orientation", ["col", "row"])
@pytest.mark.parametrize("p,r,N", [(50, 5, 450), (200, 20, 100), (37, 3, 33),
                                   (128, 16, 32), (200, 24, 65), (64, 8, 1)])
def test_filter_matches_oracle(orientation, p, r, N):
    A, X = _problem(1000 + p + N, p, r, N)
    Zg, it = _run(A, X, orientation)
    ref = l1filter.adm_l1(X, A)
    assert np.all(np.isfinite(Zg))
    assert relerr(A @ Zg, A @ ref.Z) < TOL
    # every column: the recovered column agrees too
    colerr = np.linalg.norm(A @ (Zg - ref.Z), axis=0) / \
        np.maximum(np.linalg.norm(A @ ref.Z, axis=0), 1e-30)
    assert colerr.max() < 10 * TOL
    assert (it > 0).all()


def test_filter_zero_and_clean_columns():
    rng = np.random.default_rng(7)
    p, r, N = 60, 4, 40
    A, _ = np.linalg.qr(rng.standard_normal((p, r)))
    A = A.astype(np.float32).astype(np.float64)
    X = (A @ rng.standard_normal((r, N))).astype(np.float32).astype(np.float64)
    X[:, 3] = 0.0
    X[:, 17] = 0.0
    Zg, it = _run(A, X, "col")
    assert np.all(Zg[:, [3, 17]] == 0.0)
    assert it[3] == 0 and it[17] == 0
    # uncorrupted columns: least squares after one iteration (Algorithm 1
    # with beta_0 = 1/||x||_inf makes the first shrinkage zero)
    mask = np.ones(N, bool)
    mask[[3, 17]] = False
    np.testing.assert_array_equal(it[mask], 1)
    assert relerr(Zg[:, mask], A.T @ X[:, mask]) < 1e-6


def test_filter_rank_cap_and_scale():
    # columns past *d_rank are written as zero; d_scale multiplies z
    A, X = _problem(11, 80, 8, 70)
    sc = np.linspace(0.5, 2.0, 8)
    Zg, _ = _run(A, X, "row", rank=8, scale=sc)
    ref = l1filter.adm_l1(X, A)
    assert relerr(Zg / sc[:, None], ref.Z) < TOL
    Zr, _ = _run(A[:, :5], X, "col")  # reference for a rank-5 basis
    A5 = np.hstack([A[:, :5], np.zeros((80, 3))])
    Zc, _ = _run(A5, X, "col", rank=5)
    assert np.all(Zc[5:] == 0.0)
    np.testing.assert_allclose(Zc[:5], Zr, rtol=0, atol=1e-6 * np.abs(Zr).max())


def test_filter_max_iter_flags_unconverged():
    A, X = _problem(12, 100, 10, 40, dens=0.2)
    Zg, it = _run(A, X, "col", max_iter=2)
    assert (it == -2).all()
    assert np.all(np.isfinite(Zg))


def test_filter_deterministic():
    A, X = _problem(13, 150, 12, 96)
    z1, _ = _run(A, X, "row")
    z2, _ = _run(A, X, "row")
    np.testing.assert_array_equal(z1, z2)
