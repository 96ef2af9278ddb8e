"""GPU tests of the serving loop (pcp_serve_*): continuous batching.

Requests of uneven sizes are submitted without blocking; the scheduler
admits them by device-memory footprint and slot count and runs admitted
groups as batched solves on several streams, overlapping on the device.
Checked through the C ABI: each served result equals the same request
solved alone (a batch of one) bit for bit, matches the FP64 oracle within
1e-5, requests over the budget are refused with PCP_ERR_NOMEM, poll reports
PCP_ERR_BUSY while pending, and stop cancels requests not yet launched.
"""
import time

import numpy as np
import pytest

from oracle import l1filter
from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, relerr, to_dev_cm

pytestmark = pytest.mark.gpu

TOL = 1e-5
PCP_ERR_NOMEM, PCP_ERR_BUSY, PCP_ERR_CANCELLED = -2, -8, -10


def _instances(count=8, seed=23):
    return synth.uneven_instances(count=count, seed=seed, m_range=(300, 1500),
                                  n_range=(250, 1300), r_max=12)


def _prob(P):
    import paper_1108_5359_gb300 as pk
    dM = to_dev_cm(P.M.astype(np.float32))
    Lu = pk.colmajor(P.m, P.r, fill=0.0)
    Lv = pk.colmajor(P.n, P.r, fill=0.0)
    S = pk.colmajor(P.m, P.n, fill=0.0)
    q = pk.problem(pk.pcp_params_default(P.m, P.n, P.r), dM, Lu, Lv, S,
                   P.rows, P.cols)
    return q, (Lu, Lv, S)


def _host(bufs):
    return [b.cpu().numpy() for b in bufs]


def _alone(P):
    import torch
    import paper_1108_5359_gb300 as pk
    q, bufs = _prob(P)
    st, infos = pk.pcp_l1filter_batch([q], raise_on_error=False)
    torch.cuda.synchronize()
    return st, _host(bufs)


def test_served_mix_equals_alone_and_oracle():
    import paper_1108_5359_gb300 as pk
    build_and_load()
    Ps = _instances()
    srv = pk.Server(hbm_budget_bytes=4 << 30, max_slots=64, streams=4)
    subs = []
    for i, P in enumerate(Ps):
        q, bufs = _prob(P)
        subs.append((srv.submit(q), bufs))
        if i % 3 == 2:
            time.sleep(0.002)   # later arrivals join while earlier ones run
    res = [srv.wait(t) for t, _ in subs]
    srv.close()
    for i, (P, (st, inf), (_, bufs)) in enumerate(zip(Ps, res, subs)):
        st1, ref = _alone(P)
        assert st == st1 == inf.status, i
        for a, b in zip(_host(bufs), ref):
            np.testing.assert_array_equal(a, b)
        assert inf.t_total_ms > 0
    i = min(range(len(Ps)), key=lambda i: Ps[i].m * Ps[i].n)
    P = Ps[i]
    Lu, Lv, S = (x.astype(np.float64) for x in _host(subs[i][1]))
    M = P.M.astype(np.float32).astype(np.float64)
    ref = l1filter.l1_filter_pcp(M, P.rows, P.cols, r=P.r)
    if ref.rank == P.r and res[i][0] == 0:
        assert relerr(Lu @ Lv.T, ref.L) < TOL
        assert relerr(S, ref.S) < TOL


def test_budget_refusal_and_busy_poll():
    import paper_1108_5359_gb300 as pk
    build_and_load()
    # a recoverable instance (rank test passes): 901 x 1009, rank 6
    P = synth.uneven_instances(count=6, seed=11, m_range=(300, 1400),
                               n_range=(250, 1200), r_max=12, indices=[1])[0]
    srv = pk.Server(hbm_budget_bytes=64 << 10, max_slots=4, streams=1)
    q, _ = _prob(P)
    t = srv.submit(q)
    st, inf = srv.wait(t)
    assert st == PCP_ERR_NOMEM and inf.status == PCP_ERR_NOMEM
    srv.close()
    srv = pk.Server(hbm_budget_bytes=1 << 30, max_slots=4, streams=1)
    q, _ = _prob(P)
    t = srv.submit(q)
    seen = []
    deadline = time.time() + 60
    while time.time() < deadline:
        st, inf = srv.poll(t)
        seen.append(st)
        if st != PCP_ERR_BUSY:
            break
        time.sleep(0.0005)
    assert seen[0] == PCP_ERR_BUSY
    assert seen[-1] == 0 and inf.status == 0
    st, _ = srv.poll(t)             # released after completion
    assert st == -1
    srv.close()


def test_stop_cancels_queued_requests():
    import paper_1108_5359_gb300 as pk
    build_and_load()
    Ps = _instances(count=6, seed=31)
    srv = pk.Server(hbm_budget_bytes=4 << 30, max_slots=1, streams=1)
    tickets = []
    keep = []
    for P in Ps:
        q, bufs = _prob(P)
        keep.append((q, bufs))
        tickets.append(srv.submit(q))
    srv.stop()
    sts = [srv.poll(t)[0] for t in tickets]
    assert PCP_ERR_BUSY not in sts
    assert sts.count(PCP_ERR_CANCELLED) >= 1
    assert all(s in (0, PCP_ERR_CANCELLED) or s < 0 for s in sts)
    with pytest.raises(pk.PCPError):
        srv.submit(keep[0][0])
    srv.close()


def test_served_request_grows_its_seed():
    # a request whose 50 x 50 seed fails Eq. rank_test goes back to the head
    # of the queue with the grown seed (Section 3.5) and completes
    import paper_1108_5359_gb300 as pk
    from tests.gpuhelp import to_host
    from tests.test_gpu_grow import _instance
    build_and_load()
    M, L0, S0, ro, co = _instance(0)
    m, n = M.shape
    dM = to_dev_cm(M.astype(np.float32))
    Lu, Lv, S = pk.colmajor(m, 5), pk.colmajor(n, 5), pk.colmajor(m, n)
    p = pk.pcp_params_default(m, n, 5)
    p.grow_seed = 1
    q = pk.problem(p, dM, Lu, Lv, S, row_order=ro, col_order=co)
    srv = pk.Server(hbm_budget_bytes=1 << 30, max_slots=4, streams=2)
    st, inf = srv.wait(srv.submit(q))
    srv.close()
    assert st == 0 and inf.seed_m > 50 and inf.rank == 5
    L = to_host(Lu) @ to_host(Lv).T
    assert relerr(L, L0) < TOL


def test_served_growth_that_gives_up_still_writes_the_outputs():
    # the growth of a full-rank Gaussian matrix's 30 x 30 seed gives up
    # (Section 3.5): the served request ends with PCP_ERR_RANK_TEST and the
    # outputs a batch of one without growth writes, bit for bit
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    rng = np.random.default_rng(5)
    M = rng.standard_normal((300, 280))
    ro, co = rng.permutation(300), rng.permutation(280)
    outs = []
    for grow in (True, False):
        dM = to_dev_cm(M.astype(np.float32))
        bufs = (pk.colmajor(300, 3, fill=0.0), pk.colmajor(280, 3, fill=0.0),
                pk.colmajor(300, 280, fill=0.0))
        p = pk.pcp_params_default(300, 280, 3)
        p.grow_seed = 1 if grow else 0
        q = pk.problem(p, dM, *bufs, row_order=ro, col_order=co)
        if grow:
            srv = pk.Server(hbm_budget_bytes=1 << 30, max_slots=4, streams=2)
            st, inf = srv.wait(srv.submit(q))
            srv.close()
        else:
            st, infs = pk.pcp_l1filter_batch([q], raise_on_error=False)
            torch.cuda.synchronize()
        assert st == -5
        outs.append(_host(bufs))
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
