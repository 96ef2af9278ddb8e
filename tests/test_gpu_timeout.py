"""Failure detection on the GPU without a fault: a bounded device wait runs
out, the kernel reports it, and the device stays usable.

The seed PCP's cooperative grid separates the phases of every ALM iteration
with a software grid barrier whose wait is bounded by pcp_params
.wait_timeout_ns.  Here the limit is 1 ns: waits in a 152-CTA grid last far
longer, so the first CTA that has to wait gives up, raises the solve's error
word, every other CTA leaves at its next barrier, and the call returns
PCP_ERR_TIMEOUT.  A normal solve in the same process afterwards must still
match the FP64 oracle (the context was not lost).  (The S pass's bounded
mbarrier waits are not made to run out here; see the design notes.)
"""
import numpy as np
import pytest

from oracle import l1filter
from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu


def _solve(pk, P, dM, **kw):
    import torch
    p = pk.pcp_params_default(P.m, P.n, P.r)
    for k, v in kw.items():
        setattr(p, k, v)
    plan = pk.Plan(p, P.rows, P.cols)
    Lu, Lv = pk.colmajor(P.m, P.r), pk.colmajor(P.n, P.r)
    S = pk.colmajor(P.m, P.n)
    st, info, _, _ = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, S,
                                           raise_on_error=False)
    torch.cuda.synchronize()
    plan.close()
    return st, info, Lu, Lv, S


def test_seed_barrier_wait_runs_out_and_device_recovers():
    import paper_1108_5359_gb300 as pk
    from paper_1108_5359_gb300 import _abi
    build_and_load()
    P = synth.make_config("c2_5000_r20", seed=0, m=1200, n=1100)
    M32 = P.M.astype(np.float32)
    dM = to_dev_cm(M32)
    # the grid form of the seed (152 CTAs, software barrier), 1 ns per wait
    st, info, *_ = _solve(pk, P, dM, wait_timeout_ns=1, seed_ctas=152)
    assert st == _abi.PCP_ERR_TIMEOUT, (st, pk._abi.last_error())
    assert info.status == _abi.PCP_ERR_TIMEOUT
    assert "timed out" in pk._abi.last_error()
    # the same process, the same device: a normal solve is exact
    st, info, Lu, Lv, S = _solve(pk, P, dM, seed_ctas=152)
    assert st == 0
    ref = l1filter.l1_filter_pcp(M32.astype(np.float64), P.rows, P.cols,
                                 r=P.r)
    L = to_host(Lu) @ to_host(Lv).T
    assert relerr(L, ref.L) < 1e-5
    assert relerr(to_host(S), ref.S) < 1e-5
