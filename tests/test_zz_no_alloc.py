"""The allocation-free seed PCP entry point matches the workspace one.

pcp_seed_pcp_static is for callers that cannot call cudaMalloc (their host
framework owns all device memory, or an allocation's implicit device
synchronisation is not acceptable where they run): its scratch is a fixed
device array owned by the library instead of a caller buffer.  This file
runs last so that a failure here leaves every other test already run.

Checked through the C ABI: two calls in a row on different seeds (so the
second call starts from the first call's leftover scratch) give bit for bit
the same U^s, Sigma^s, V^s, rank, iteration count and residual as
pcp_seed_pcp with its own workspace.  Both run the same kernel on the same
input, and the seed's reductions sum fixed partial-sum slots in a fixed
order, so any difference would come from state left in the shared array by
the previous call.  An oversized seed is refused with a clear error before
any device work.
"""
import numpy as np
import pytest

from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, to_dev_cm, to_host

pytestmark = pytest.mark.gpu

def _k(mp, np_, r):
    k0 = min((r + max(6, r // 4) + 1) // 2 * 2, min(mp, np_) // 2 * 2)
    kmax = min(min(mp, np_) // 2 * 2, max(k0 + 16, 2 * k0) // 2 * 2, 64)
    return k0, kmax


def _outputs(mp, np_, kmax):
    import torch
    U = torch.zeros((kmax, mp), dtype=torch.float64, device="cuda").t()
    V = torch.zeros((kmax, np_), dtype=torch.float64, device="cuda").t()
    S = torch.zeros(kmax, dtype=torch.float64, device="cuda")
    return U, S, V


def _seed_problem(cfg, seed, **kw):
    P = synth.make_config(cfg, seed=seed, **kw)
    D = P.M[np.ix_(P.rows, P.cols)].astype(np.float32).astype(np.float64)
    return D, P.r


def _args(D, r):
    mp, np_ = D.shape
    k0, kmax = _k(mp, np_, r)
    lam = 1.0 / np.sqrt(max(mp, np_))
    return dict(lam=lam, tol=1e-7, rho=1.5, mu_scale=1.25, mu_max_ratio=1e7,
                max_iter=500, k0=k0, kmax=kmax, rank_cut=1e-6, r_cap=r)


def test_static_matches_workspace_two_calls_in_a_row():
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    cases = [_seed_problem("c2_5000_r20", 0, m=1200, n=1100),
             _seed_problem("c1_500_r5", 3)]
    static_out = []
    for D, r in cases:  # back to back: the second reuses the first's scratch
        a = _args(D, r)
        U, S, V = _outputs(D.shape[0], D.shape[1], a["kmax"])
        st, rank, iters, res = pk.pcp_seed_pcp_static(
            to_dev_cm(D), a["lam"], a["tol"], a["rho"], a["mu_scale"],
            a["mu_max_ratio"], a["max_iter"], a["k0"], a["kmax"],
            a["rank_cut"], a["r_cap"], U, S, V)
        torch.cuda.synchronize()
        static_out.append((st, rank, iters, res,
                           (to_host(U), to_host(S), to_host(V))))
    for (D, r), (st, rank, iters, res, outs) in zip(cases, static_out):
        a = _args(D, r)
        U, S, V = _outputs(D.shape[0], D.shape[1], a["kmax"])
        work = torch.empty(pk.pcp_seed_workspace_bytes(D.shape[0], D.shape[1],
                                                       a["kmax"]),
                           dtype=torch.uint8, device="cuda")
        st2, rank2, iters2, res2 = pk.pcp_seed_pcp(
            to_dev_cm(D), a["lam"], a["tol"], a["rho"], a["mu_scale"],
            a["mu_max_ratio"], a["max_iter"], a["k0"], a["kmax"],
            a["rank_cut"], a["r_cap"], work, U, S, V)
        torch.cuda.synchronize()
        assert st == st2 == 0
        assert rank == rank2 == r
        assert iters == iters2
        assert res == res2 and res <= 1e-7
        for got, want in zip(outs, (to_host(U), to_host(S), to_host(V))):
            np.testing.assert_array_equal(got, want)


def test_static_refuses_oversized_seed():
    import ctypes as C
    from paper_1108_5359_gb300 import _abi
    lib = build_and_load()
    rank = C.c_int32()
    st = lib.pcp_seed_pcp_static(None, 256, 256, 0.0, 1e-7, 1.5, 1.25, 1e7,
                                 10, 8, 64, 1e-10, 0, None, None, None,
                                 C.byref(rank), None, None, None)
    assert st == _abi.PCP_ERR_ARG
    msg = lib.pcp_last_error().decode()
    assert "needs" in msg and "more than the fixed" in msg
