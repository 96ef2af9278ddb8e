"""GPU parity of the seed stage: gather (Eq. partition) and the FP64 seed PCP
(Eq. SPCP by inexact ALM with SVT).

The device ALM uses a partial SVD (subspace iteration + Rayleigh-Ritz) where
the oracle uses a full LAPACK SVD; both stop at ||D-L-S||_F/||D||_F <= 1e-7,
so the recovered L^s agree to the level of that tolerance (1e-6 relative is
asserted).  Also checked: rank, U^s and V^s orthonormal to FP64 rounding
(1e-12), the sorted singular values, exact recovery of L0^s, the zero seed,
the gather being exact, and the same bits from every team form (grid sizes,
thread-block clusters).
"""
import numpy as np
import pytest

from oracle import pcp
from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, idx_dev, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu


def _seed(D, r, kmax=None, tol=1e-7, lam=None, k0=None):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    mp, np_ = D.shape
    k0 = k0 or min((r + max(6, r // 4) + 1) // 2 * 2, min(mp, np_) // 2 * 2)
    kmax = kmax or min(min(mp, np_) // 2 * 2, max(k0 + 16, 2 * k0) // 2 * 2, 64)
    work = torch.empty(pk.pcp_seed_workspace_bytes(mp, np_, kmax),
                       dtype=torch.uint8, device="cuda")
    dD = to_dev_cm(D)
    U = torch.zeros((kmax, mp), dtype=torch.float64, device="cuda").t()
    V = torch.zeros((kmax, np_), dtype=torch.float64, device="cuda").t()
    Sg = torch.zeros(kmax, dtype=torch.float64, device="cuda")
    lam = lam or 1.0 / np.sqrt(max(mp, np_))
    st, rank, iters, res = pk.pcp_seed_pcp(dD, lam, tol, 1.5, 1.25, 1e7, 500,
                                           k0, kmax, 1e-6, r, work, U, Sg, V)
    torch.cuda.synchronize()
    return to_host(U), to_host(Sg), to_host(V), rank, iters, res


@pytest.mark.parametrize("cfg,seed", [("c1_500_r5", 3), ("c1_500_r5", 4),
                                      ("c2_5000_r20", 0)])
def test_seed_pcp_matches_oracle(cfg, seed):
    if cfg.startswith("c2"):
        P = synth.make_config(cfg, seed=seed, m=1200, n=1100)
    else:
        P = synth.make_config(cfg, seed=seed)
    D = P.M[np.ix_(P.rows, P.cols)].astype(np.float32).astype(np.float64)
    lam = 1.0 / np.sqrt(max(D.shape))
    ref = pcp.inexact_alm_pcp(D, lam)
    U, s, V, rank, iters, res = _seed(D, P.r)
    assert rank == P.r == ref.sigma.size
    assert res <= 1e-7
    Lg = (U[:, :rank] * s[:rank]) @ V[:, :rank].T
    assert relerr(Lg, ref.L) < 1e-6
    L0s = P.L0[np.ix_(P.rows, P.cols)]
    assert relerr(Lg, L0s) < 1e-5
    # Algorithm 1 (step 2, Eq. l1g) takes A^T A = I: the seed's bases are
    # orthonormal to FP64 rounding (the final FP64 skinny SVD)
    np.testing.assert_allclose(U[:, :rank].T @ U[:, :rank], np.eye(rank),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(V[:, :rank].T @ V[:, :rank], np.eye(rank),
                               rtol=0, atol=1e-12)
    assert np.all(np.diff(s[:rank]) <= 0)
    np.testing.assert_allclose(s[:rank], np.sort(ref.sigma)[::-1], rtol=1e-6)
    assert np.all(U[:, rank:] == 0) and np.all(s[rank:] == 0)
    assert abs(iters - ref.iters) <= 5


def test_seed_pcp_ragged_small():
    M, L0, S0 = synth.lowrank_plus_sparse(46, 38, 3, 0.05, -20, 20, seed=21)
    ref = pcp.inexact_alm_pcp(M, 1.0 / np.sqrt(46))
    U, s, V, rank, iters, res = _seed(M, 3)
    assert rank == ref.sigma.size == 3
    Lg = (U[:, :rank] * s[:rank]) @ V[:, :rank].T
    assert relerr(Lg, ref.L) < 1e-6


def test_seed_pcp_zero_matrix():
    U, s, V, rank, iters, res = _seed(np.zeros((20, 20)), 2)
    assert rank == 0 and np.all(U == 0) and np.all(s == 0)


def test_gather_is_exact():
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    rng = np.random.default_rng(5)
    M = rng.standard_normal((301, 257)).astype(np.float32)
    rows = np.sort(rng.choice(301, 40, replace=False))
    cols = np.sort(rng.choice(257, 33, replace=False))
    dM = to_dev_cm(M, ld=305)
    out = torch.zeros((33, 40), dtype=torch.float64, device="cuda").t()
    pk.pcp_gather_seed(dM, idx_dev(rows), idx_dev(cols), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_host(out),
                                  M[np.ix_(rows, cols)].astype(np.float64))


@pytest.mark.parametrize("cfg,kw", [("c1_500_r5", {}),
                                    ("c2_5000_r20", dict(m=1200, n=1100))])
def test_seed_result_does_not_depend_on_team(cfg, kw):
    # every team form sums the same fixed partial-sum slots in the same
    # order, so a cooperative grid of any size (0 = library choice, 24, 57
    # CTAs) and one thread-block cluster (8 or 16 CTAs, hardware barrier)
    # give bit-identical factors
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P = synth.make_config(cfg, seed=3, **kw)
    dM = to_dev_cm(P.M.astype(np.float32))
    outs = []
    for ctas in (0, 24, 57, 8, 16):
        p = pk.pcp_params_default(P.m, P.n, P.r)
        p.seed_ctas = ctas
        plan = pk.Plan(p, P.rows, P.cols)
        Lu, Lv = pk.colmajor(P.m, P.r), pk.colmajor(P.n, P.r)
        st, info, _, _ = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, None)
        torch.cuda.synchronize()
        plan.close()
        outs.append((Lu.cpu().numpy(), Lv.cpu().numpy(), info.seed_iters))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2]


def test_seed_pcp_at_the_largest_side_and_subspace():
    # the largest seed the stage takes (512 x 512) with the largest subspace
    # (k0 = 60 for rank 48, growing to kmax = 64): the blocked k x k
    # Cholesky and every per-side loop at its bound
    M, L0, S0 = synth.lowrank_plus_sparse(512, 512, 48, 0.05, -30, 30,
                                          seed=31)
    lam = 1.0 / np.sqrt(512)
    ref = pcp.inexact_alm_pcp(M, lam)
    U, s, V, rank, iters, res = _seed(M, 48)
    assert U.shape == (512, 64)
    assert rank == ref.sigma.size == 48
    assert res <= 1e-7
    Lg = (U[:, :rank] * s[:rank]) @ V[:, :rank].T
    assert relerr(Lg, ref.L) < 1e-6
    assert relerr(Lg, L0) < 1e-5
    np.testing.assert_allclose(U[:, :rank].T @ U[:, :rank], np.eye(rank),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(s[:rank], np.sort(ref.sigma)[::-1], rtol=1e-6)
    assert np.all(U[:, rank:] == 0) and np.all(s[rank:] == 0)


def test_seed_pcp_skinny_at_the_widest_subspace():
    # 512 x 41 seed of rank 2 + 3% outliers (exactly recovered by PCP): the
    # short side is odd, so the widest subspace the entry point takes is
    # kmax = 40 (even, <= 41), here from the first step (k0 = 40); most CTAs
    # own no column of the short side.  (A subspace wider than the short
    # side is refused: its extra vector's Cholesky pivot is FP32 rounding
    # noise, not zero, and on a 512 x 7 seed with kmax = 8 the noise column
    # moved L by 3.6e-4.)
    M, L0, S0 = synth.lowrank_plus_sparse(512, 41, 2, 0.03, -10, 10, seed=32)
    lam = 1.0 / np.sqrt(512)
    ref = pcp.inexact_alm_pcp(M, lam)
    U, s, V, rank, iters, res = _seed(M, 2, kmax=40, k0=40)
    assert rank == ref.sigma.size == 2
    assert res <= 1e-7
    Lg = (U[:, :rank] * s[:rank]) @ V[:, :rank].T
    assert relerr(Lg, ref.L) < 1e-6
    assert relerr(Lg, L0) < 1e-6
    np.testing.assert_allclose(s[:rank], np.sort(ref.sigma)[::-1], rtol=1e-6)
    np.testing.assert_allclose(V[:, :rank].T @ V[:, :rank], np.eye(rank),
                               rtol=0, atol=1e-12)
    assert np.all(U[:, rank:] == 0) and np.all(V[:, rank:] == 0)
