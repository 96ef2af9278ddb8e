"""GPU parity of the S pass (S = M - Lu Lv^T, Algorithm 2 output).

Against an FP64 NumPy product on the same FP32 inputs; tolerance is FP32
rounding of an r-term dot product.  Ragged m, n (tile tails), r from 0 to 64,
leading dimensions that break 16-byte alignment (scalar path) and the
in-place form S = M.
"""
import numpy as np
import pytest

from tests.gpuhelp import build_and_load, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu


def _case(m, n, r, ldm=None, lds=None, seed=0, inplace=False):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((m, n)).astype(np.float32) * 10
    Lu = rng.standard_normal((m, r)).astype(np.float32)
    Lv = rng.standard_normal((n, r)).astype(np.float32)
    dM = to_dev_cm(M, ld=ldm)
    dLu = to_dev_cm(Lu) if r else torch.zeros((1, m), device="cuda").t()[:, :0]
    dLv = to_dev_cm(Lv) if r else torch.zeros((1, n), device="cuda").t()[:, :0]
    dS = dM if inplace else to_dev_cm(np.full((m, n), np.nan, np.float32),
                                      ld=lds)
    pk.pcp_spass(dM, dLu, dLv, dS)
    torch.cuda.synchronize()
    ref = M.astype(np.float64) - Lu.astype(np.float64) @ Lv.astype(np.float64).T
    return to_host(dS), ref, r


@pytest.mark.parametrize("m,n,r", [(128, 64, 5), (500, 500, 5), (1000, 777, 20),
                                   (131, 67, 1), (5, 3, 2), (300, 200, 50),
                                   (256, 128, 64), (64, 64, 0)])
def test_spass_matches_fp64(m, n, r):
    S, ref, r = _case(m, n, r)
    err = np.abs(S - ref).max()
    bound = 4 * np.finfo(np.float32).eps * (10 * 4 + 2 * max(r, 1) * 4)
    assert err <= bound * np.sqrt(max(r, 1)), err


def test_spass_unaligned_leading_dims():
    S, ref, _ = _case(301, 97, 7, ldm=303, lds=305)
    assert relerr(S, ref) < 1e-6


def test_spass_in_place():
    S, ref, _ = _case(256, 130, 9, inplace=True)
    assert relerr(S, ref) < 1e-6


def test_spass_large_ragged():
    S, ref, _ = _case(4099, 1031, 20, seed=3)
    assert relerr(S, ref) < 1e-6


@pytest.mark.parametrize("m,n,r,ldm,lds,inplace", [
    (4099, 1031, 50, None, None, False),   # ragged tails
    (301, 97, 40, 303, 305, False),        # odd leading dimensions
    (256, 130, 64, None, None, True),      # in place
    (129, 33, 33, None, None, False)])
def test_spass_high_rank(m, n, r, ldm, lds, inplace):
    # ranks above 32 (the 20000 x 20000 rank-50 workload's range)
    S, ref, r = _case(m, n, r, ldm=ldm, lds=lds, seed=r, inplace=inplace)
    err = np.abs(S - ref).max()
    bound = 4 * np.finfo(np.float32).eps * (10 * 4 + 2 * r * 4)
    assert err <= bound * np.sqrt(r), err
    assert relerr(S, ref) < 1e-6
