"""GPU parity of pcp_l1filter_solve_host (Algorithm 2 on host buffers, the
copies overlapped with the compute).

The host-buffer solve runs the same kernels as the device-buffer solve on
the same seed, so the factors must agree bit for bit; S agrees to FP32
rounding (its column chunks may end in a narrow chunk that the S pass
computes with the FP32 FMA kernel instead of the tensor cores).  Covered:
page-locked and pageable M, a leading dimension larger than m for M and S,
factors only, the asynchronous form (no info), and seed growth (Section
3.5) starting from host buffers.
"""
import numpy as np
import pytest

from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu


def _host_cm(a, ld=None, pin=True):
    import torch
    rows, cols = a.shape
    ld = ld or rows
    buf = torch.zeros((cols, ld), dtype=torch.float32)
    if pin:
        buf = buf.pin_memory()
    buf[:, :rows] = torch.from_numpy(np.ascontiguousarray(a.T, np.float32))
    return buf.t()[:rows, :]


def _device_solve(P, M32):
    import torch
    import paper_1108_5359_gb300 as pk
    p = pk.pcp_params_default(P.m, P.n, P.r)
    plan = pk.Plan(p, P.rows, P.cols)
    dM = to_dev_cm(M32)
    Lu, Lv, S = pk.colmajor(P.m, P.r), pk.colmajor(P.n, P.r), \
        pk.colmajor(P.m, P.n)
    st, info, _, _ = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, S)
    torch.cuda.synchronize()
    plan.close()
    return to_host(Lu), to_host(Lv), to_host(S)


@pytest.mark.parametrize("shape,pin,ldm,lds", [
    ((500, 500, 5), True, None, None),
    ((1203, 961, 9), True, 1208, 1211),
    ((1203, 961, 9), False, None, None)])
def test_host_solve_matches_device_solve(shape, pin, ldm, lds):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    m, n, r = shape
    P = synth.make_config("c1_500_r5", seed=4, m=m, n=n, r=r)
    M32 = P.M.astype(np.float32)
    Lu_d, Lv_d, S_d = _device_solve(P, M32)
    hM = _host_cm(M32, ld=ldm, pin=pin)
    hLu = _host_cm(np.zeros((m, r)), pin=pin)
    hLv = _host_cm(np.zeros((n, r)), pin=pin)
    hS = _host_cm(np.full((m, n), np.nan), ld=lds, pin=pin)
    p = pk.pcp_params_default(m, n, r)
    plan = pk.Plan(p, P.rows, P.cols)
    for _ in range(2):  # the second call reuses the plan's device buffers
        st, info = pk.pcp_l1filter_solve_host(plan, hM, hLu, hLv, hS)
        assert st == 0 and info.status == 0
        np.testing.assert_array_equal(hLu.numpy(), Lu_d)
        np.testing.assert_array_equal(hLv.numpy(), Lv_d)
        assert relerr(hS.numpy().astype(np.float64), S_d) < 1e-6
    plan.close()
    L = Lu_d @ Lv_d.T
    assert relerr(L, P.L0) < 1e-5


def test_host_solve_factors_only_and_async():
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P = synth.make_config("c1_500_r5", seed=5)
    M32 = P.M.astype(np.float32)
    Lu_d, Lv_d, _ = _device_solve(P, M32)
    hM = _host_cm(M32)
    hLu, hLv = _host_cm(np.zeros((P.m, P.r))), _host_cm(np.zeros((P.n, P.r)))
    plan = pk.Plan(pk.pcp_params_default(P.m, P.n, P.r), P.rows, P.cols)
    st, inf = pk.pcp_l1filter_solve_host(plan, hM, hLu, hLv, None, info=False)
    assert st == 0 and inf is None
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hLu.numpy(), Lu_d)
    np.testing.assert_array_equal(hLv.numpy(), Lv_d)
    plan.close()


def test_host_solve_grows_the_seed():
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    M, L0, S0 = synth.lowrank_plus_sparse(600, 560, 5, 0.12, -50, 50,
                                          seed=(0, 77))
    rng = np.random.default_rng(0)
    ro, co = rng.permutation(600), rng.permutation(560)
    M32 = M.astype(np.float32)
    p = pk.pcp_params_default(600, 560, 5)
    p.grow_seed = 1
    plan = pk.Plan(p, row_order=ro, col_order=co)
    hM = _host_cm(M32)
    hLu, hLv = _host_cm(np.zeros((600, 5))), _host_cm(np.zeros((560, 5)))
    hS = _host_cm(np.zeros((600, 560)))
    st, info = pk.pcp_l1filter_solve_host(plan, hM, hLu, hLv, hS,
                                          raise_on_error=False)
    torch.cuda.synchronize()
    plan.close()
    assert st == 0, info.as_dict()
    assert info.seed_m > 50 and info.seed_n > 50
    L = hLu.numpy().astype(np.float64) @ hLv.numpy().astype(np.float64).T
    assert relerr(L, L0) < 1e-5
    assert relerr(hS.numpy().astype(np.float64), S0) < 1e-5


def test_async_solves_replay_a_graph_with_the_same_results():
    # without info the second call with the same buffers is captured into a
    # CUDA graph and later calls replay it; new buffers are captured anew
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P = synth.make_config("c1_500_r5", seed=6, m=900, n=700, r=6)
    M32 = P.M.astype(np.float32)
    Lu_d, Lv_d, S_d = _device_solve(P, M32)
    plan = pk.Plan(pk.pcp_params_default(P.m, P.n, P.r), P.rows, P.cols)
    dM = to_dev_cm(M32)
    for bufset in range(2):
        Lu, Lv = pk.colmajor(P.m, P.r), pk.colmajor(P.n, P.r)
        S = pk.colmajor(P.m, P.n)
        for _ in range(4):
            Lu.fill_(float("nan"))
            S.fill_(float("nan"))
            st, inf, _, _ = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, S,
                                                  info=False)
            assert st == 0 and inf is None
            torch.cuda.synchronize()
            np.testing.assert_array_equal(to_host(Lu), Lu_d)
            np.testing.assert_array_equal(to_host(Lv), Lv_d)
            np.testing.assert_array_equal(to_host(S), S_d)
    # calls 2..4 of the first buffer set and 1..4 of the second replayed
    assert pk.pcp_plan_graph_launches(plan) == 7
    # host buffers, asynchronous, replayed
    hM = _host_cm(M32)
    hLu, hLv = _host_cm(np.zeros((P.m, P.r))), _host_cm(np.zeros((P.n, P.r)))
    hS = _host_cm(np.zeros((P.m, P.n)))
    for _ in range(4):
        hS.fill_(float("nan"))
        st, _ = pk.pcp_l1filter_solve_host(plan, hM, hLu, hLv, hS, info=False)
        assert st == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hLu.numpy(), Lu_d)
        np.testing.assert_array_equal(hLv.numpy(), Lv_d)
        assert relerr(hS.numpy().astype(np.float64), S_d) < 1e-6
    assert pk.pcp_plan_graph_launches(plan) == 11
    plan.close()


def test_pageable_host_buffers_give_the_same_results():
    # pageable memory: the seed cannot read M in place and the copies are
    # synchronous for the host; whether the CUDA driver captures them into the
    # graph (replays) or not (graphs off, -1), the results are the same
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P = synth.make_config("c1_500_r5", seed=6, m=700, n=520, r=6)
    M32 = P.M.astype(np.float32)
    Lu_d, Lv_d, S_d = _device_solve(P, M32)
    plan = pk.Plan(pk.pcp_params_default(P.m, P.n, P.r), P.rows, P.cols)
    hM = _host_cm(M32, pin=False)
    hLu = _host_cm(np.zeros((P.m, P.r)), pin=False)
    hLv = _host_cm(np.zeros((P.n, P.r)), pin=False)
    hS = _host_cm(np.zeros((P.m, P.n)), pin=False)
    for _ in range(3):
        st, _ = pk.pcp_l1filter_solve_host(plan, hM, hLu, hLv, hS, info=False)
        assert st == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hLu.numpy(), Lu_d)
        np.testing.assert_array_equal(hLv.numpy(), Lv_d)
        assert relerr(hS.numpy().astype(np.float64), S_d) < 1e-6
    assert pk.pcp_plan_graph_launches(plan) in (-1, 2)
    plan.close()
