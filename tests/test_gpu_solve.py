"""GPU parity of the whole path (Algorithm 2) through pcp_l1filter_solve.

Seed PCP (FP64) -> column and row filtering (FP32 Algorithm 1) -> factor
assembly (Eq. l1s') -> S = M - L.  The GPU's L = Lu Lv^T and S must match
the FP64 oracle within relative Frobenius error 1e-5 on the same input and
the same seed index sets; on recoverable inputs both recover L0 and S0.
Sizes span several tiles with ragged tails; the largest case is the
5000 x 5000, rank-20 workload (seed 200 x 200, 10% corruption in
[-100, 100]).
"""
import numpy as np
import pytest

from oracle import l1filter
from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _gpu_solve(P, ld=None, want_S=True, **kw):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    M32 = P.M.astype(np.float32)
    dM = to_dev_cm(M32, ld=ld)
    p = pk.pcp_params_default(P.m, P.n, P.r)
    for k, v in kw.items():
        setattr(p, k, v)
    plan = pk.Plan(p, P.rows, P.cols)
    Lu = pk.colmajor(P.m, P.r)
    Lv = pk.colmajor(P.n, P.r)
    S = pk.colmajor(P.m, P.n) if want_S else None
    st, info, rows, cols = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, S,
                                                 raise_on_error=False)
    torch.cuda.synchronize()
    plan.close()
    out = dict(st=st, info=info.as_dict(), rows=rows, cols=cols,
               Lu=to_host(Lu), Lv=to_host(Lv),
               S=to_host(S) if want_S else None,
               M=M32.astype(np.float64))
    return out


def _check(P, g, tol=TOL):
    assert g["st"] == 0, g
    np.testing.assert_array_equal(g["rows"], P.rows)
    np.testing.assert_array_equal(g["cols"], P.cols)
    ref = l1filter.l1_filter_pcp(g["M"], P.rows, P.cols, r=P.r)
    Lg = g["Lu"] @ g["Lv"].T
    assert g["info"]["rank"] == ref.rank == P.r
    assert relerr(Lg, ref.L) < tol
    if g["S"] is not None:
        assert relerr(g["S"], ref.S) < tol
        # S = M - L holds to FP32 rounding
        assert relerr(g["S"] + Lg, g["M"]) < 1e-6
    return ref, Lg


def test_solve_c1_500():
    P = synth.make_config("c1_500_r5", seed=3)
    g = _gpu_solve(P)
    ref, Lg = _check(P, g)
    assert relerr(Lg, P.L0) < TOL          # exact recovery (Section 3.4)
    assert relerr(g["S"], P.S0) < TOL
    assert g["info"]["rank_ok"] == 1
    assert g["info"]["problems"] == 900
    assert g["info"]["problems_unconverged"] == 0


def test_solve_ragged_with_leading_dim():
    P = synth.make_config("c1_500_r5", seed=5, m=437, n=389, r=4)
    g = _gpu_solve(P, ld=441)
    _check(P, g)


def test_solve_factors_only():
    P = synth.make_config("c1_500_r5", seed=5, m=300, n=650, r=3)
    g = _gpu_solve(P, want_S=False)
    _check(P, g)


def test_solve_c2_5000_full_size():
    P = synth.make_config("c2_5000_r20", seed=0)
    g = _gpu_solve(P)
    ref, Lg = _check(P, g)
    assert relerr(Lg, P.L0) < TOL
    assert relerr(g["S"], P.S0) < TOL
    # support of S recovered (threshold 1e-4 of the corruption magnitude)
    tau = 1e-2
    found = np.abs(g["S"]) > tau
    assert np.all(found[np.abs(P.S0) > 10 * tau])
    assert not np.any(found[P.S0 == 0])


def test_solve_sampled_seed_is_valid():
    # without given index sets the library samples I_s, J_s itself
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P = synth.make_config("c1_500_r5", seed=3)
    dM = to_dev_cm(P.M.astype(np.float32))
    Lu, Lv, S, info, rows, cols, st = pk.solve(dM, P.r, raise_on_error=False)
    assert len(set(rows)) == 50 and len(set(cols)) == 50
    assert np.all(np.diff(rows) > 0) and rows.min() >= 0 and rows.max() < 500
    ref = l1filter.l1_filter_pcp(P.M.astype(np.float32).astype(np.float64),
                                 rows, cols, r=P.r)
    if ref.rank == P.r and relerr(ref.L, P.L0) < 1e-6:
        assert st == 0
        assert relerr(to_host(Lu) @ to_host(Lv).T, ref.L) < TOL


def test_solve_rank_test_failure_is_reported():
    # a zero matrix has a rank-0 seed: Eq. rank_test fails, status says so
    P = synth.make_config("c1_500_r5", seed=3, m=200, n=200)
    P.M[:] = 0.0
    g = _gpu_solve(P)
    assert g["st"] == -5
    assert g["info"]["rank"] == 0
    assert np.all(g["Lu"] == 0) and np.all(g["Lv"] == 0)
    assert np.all(g["S"] == 0)


def test_solve_nonfinite_seed_is_reported():
    P = synth.make_config("c1_500_r5", seed=3, m=200, n=200)
    P.M[P.rows[2], P.cols[3]] = np.nan
    g = _gpu_solve(P, want_S=False)
    assert g["st"] == -4
