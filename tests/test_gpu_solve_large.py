"""GPU parity of the whole path at rank 50 with a 500 x 500 seed.

The 20000 x 20000 rank-50 workload (X, Y ~ N(0, 1/r), 10% corruption in
[-10, 10], seed 500 x 500) takes the paths the small workloads do not: the
seed PCP at m' = n' = 500 with a 64-wide subspace, and Algorithm 1 on the
tensor cores (p = 500 > 256, r = 50 > 32).  Checked:
  * a 3000 x 3000 instance of the same distribution against the full FP64
    oracle (relative Frobenius error 1e-5 on L and S) and against L0, S0,
    for PCP_FP32, PCP_TF32_REFINED and PCP_BF16_REFINED;
  * the full 20000 x 20000 size on a sampled 96 x 96 block of L and S, which
    the oracle computes from its own seed PCP and Algorithm 1 on just those
    rows and columns (L = Lu Lv^T is unique; the factors are not).
"""
import numpy as np
import pytest

from oracle import l1filter, pcp
from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, relerr
from tests.test_gpu_solve import _gpu_solve

pytestmark = pytest.mark.gpu

TOL = 1e-5
PCP_FP32, PCP_BF16_REFINED, PCP_TF32_REFINED = 0, 1, 2


@pytest.fixture(scope="module")
def mid():
    P = synth.make_config("c3_20000_r50", seed=0, m=3000, n=3000)
    M = P.M.astype(np.float32).astype(np.float64)
    ref = l1filter.l1_filter_pcp(M, P.rows, P.cols, r=P.r)
    return P, ref


@pytest.mark.parametrize("precision", [PCP_FP32, PCP_TF32_REFINED,
                                       PCP_BF16_REFINED])
def test_rank50_seed500_matches_oracle(mid, precision):
    P, ref = mid
    g = _gpu_solve(P, precision=precision)
    assert g["st"] == 0, g
    assert g["info"]["rank"] == ref.rank == 50
    assert g["info"]["seed_m"] == 500 and g["info"]["seed_n"] == 500
    Lg = g["Lu"] @ g["Lv"].T
    assert relerr(Lg, ref.L) < TOL
    assert relerr(g["S"], ref.S) < TOL
    assert relerr(Lg, P.L0) < TOL          # exact recovery
    assert g["info"]["problems_unconverged"] == 0


def test_rank50_full_size_sampled_block():
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P = synth.make_config("c3_20000_r50", seed=1, keep_truth=False,
                          dtype=np.float32)
    m, n, r = P.m, P.n, P.r
    dM = pk.colmajor(m, n)
    dM.copy_(torch.from_numpy(P.M))
    Lu = pk.colmajor(m, r)
    Lv = pk.colmajor(n, r)
    S = pk.colmajor(m, n)
    plan = pk.Plan(pk.pcp_params_default(m, n, r), P.rows, P.cols)
    st, info, _, _ = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, S,
                                           raise_on_error=False)
    torch.cuda.synchronize()
    plan.close()
    assert st == 0 and info.rank == 50
    rng = np.random.default_rng(5)
    rbar = np.setdiff1d(np.arange(m), P.rows)
    cbar = np.setdiff1d(np.arange(n), P.cols)
    ri = np.sort(np.concatenate([rng.choice(rbar, 80, replace=False),
                                 rng.choice(P.rows, 16, replace=False)]))
    ci = np.sort(np.concatenate([rng.choice(cbar, 80, replace=False),
                                 rng.choice(P.cols, 16, replace=False)]))
    Mh = P.M.astype(np.float64)
    # oracle: seed PCP, then Algorithm 1 on the sampled rows / columns only
    Ms = Mh[np.ix_(P.rows, P.cols)]
    seed = pcp.inexact_alm_pcp(Ms, 1.0 / np.sqrt(500.0), tol=1e-7)
    k = l1filter.numerical_rank(seed.sigma, 1e-6)
    o = np.argsort(-seed.sigma)[:min(k, r)]
    U, sig, V = seed.U[:, o], seed.sigma[o], seed.V[:, o]
    pos_r = {v: i for i, v in enumerate(P.rows)}
    pos_c = {v: i for i, v in enumerate(P.cols)}
    Lu_o = np.zeros((ri.size, r))
    Lv_o = np.zeros((ci.size, r))
    out_r = [i for i, v in enumerate(ri) if v not in pos_r]
    out_c = [i for i, v in enumerate(ci) if v not in pos_c]
    for i, v in enumerate(ri):
        if v in pos_r:
            Lu_o[i] = U[pos_r[v]]
    for i, v in enumerate(ci):
        if v in pos_c:
            Lv_o[i] = V[pos_c[v]] * sig
    rowres = l1filter.adm_l1(Mh[np.ix_(ri[out_r], P.cols)].T, V)
    colres = l1filter.adm_l1(Mh[np.ix_(P.rows, ci[out_c])], U)
    Lu_o[out_r] = rowres.Z.T / sig
    Lv_o[out_c] = colres.Z.T
    L_o = Lu_o @ Lv_o.T
    Lg = Lu.double().cpu().numpy()[ri] @ Lv.double().cpu().numpy()[ci].T
    Sg = S.double().cpu().numpy()[np.ix_(ri, ci)]
    assert relerr(Lg, L_o) < TOL
    assert relerr(Sg, Mh[np.ix_(ri, ci)] - L_o) < TOL


def test_largest_seed_512_matches_oracle():
    # the largest seed the plan takes (512 x 512) at rank 48 (k0 = 60,
    # subspace up to 64) on a 1400 x 1300 matrix of the same distribution:
    # Algorithm 1's tensor-core kernel at p = 512 on both sides
    import dataclasses
    P = synth.make_config("c3_20000_r50", seed=2, m=1400, n=1300, r=48)
    rows, cols = synth.seed_indices(P.m, P.n, 512, 512, seed=2)
    P = dataclasses.replace(P, rows=rows, cols=cols)
    g = _gpu_solve(P)
    assert g["st"] == 0, g
    assert g["info"]["seed_m"] == 512 and g["info"]["seed_n"] == 512
    ref = l1filter.l1_filter_pcp(g["M"], rows, cols, r=P.r)
    Lg = g["Lu"] @ g["Lv"].T
    assert g["info"]["rank"] == ref.rank == 48
    assert relerr(Lg, ref.L) < TOL
    assert relerr(g["S"], ref.S) < TOL
    assert relerr(Lg, P.L0) < TOL
    assert g["info"]["problems_unconverged"] == 0
