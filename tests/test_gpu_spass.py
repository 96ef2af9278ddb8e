"""GPU parity of the S pass (S = M - Lu Lv^T, Algorithm 2 output).

Against an FP64 NumPy product on the same FP32 inputs; tolerance is FP32
rounding of an r-term dot product (split-TF32 products of the tensor-core
form stay inside it).  Both kernels (FP32 SIMT; tcgen05 tensor cores with TMA
tiles) on ragged m, n (tile tails), r from 0 to 64, leading dimensions that
break 16-byte alignment (SIMT scalar path; the tensor form refuses them) and
the in-place form S = M.
"""
import numpy as np
import pytest

from tests.gpuhelp import build_and_load, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu


SIMT, TENSOR = 1, 2  # PCP_SPASS_SIMT, PCP_SPASS_TENSOR


def _tensor_ok(m, n, r, ldm=None, lds=None):
    return (r >= 1 and m >= 128 and n >= 64 and (ldm or m) % 4 == 0
            and (lds or m) % 4 == 0)


def _case(m, n, r, ldm=None, lds=None, seed=0, inplace=False, impl=None):
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
    if impl == TENSOR and not _tensor_ok(m, n, r, ldm, lds):
        pytest.skip("shape outside the tensor-core form")
    pk.pcp_spass(dM, dLu, dLv, dS, impl=impl)
    torch.cuda.synchronize()
    ref = M.astype(np.float64) - Lu.astype(np.float64) @ Lv.astype(np.float64).T
    return to_host(dS), ref, r


@pytest.mark.parametrize("impl", [None, SIMT, TENSOR])
@pytest.mark.parametrize("m,n,r", [(128, 64, 5), (500, 500, 5), (1000, 777, 20),
                                   (131, 67, 1), (5, 3, 2), (300, 200, 50),
                                   (256, 128, 64), (64, 64, 0), (129, 65, 57),
                                   (1024, 1024, 8)])
def test_spass_matches_fp64(m, n, r, impl):
    S, ref, r = _case(m, n, r, impl=impl)
    err = np.abs(S - ref).max()
    bound = 4 * np.finfo(np.float32).eps * (10 * 4 + 2 * max(r, 1) * 4)
    assert err <= bound * np.sqrt(max(r, 1)), err


def test_spass_unaligned_leading_dims():
    S, ref, _ = _case(301, 97, 7, ldm=303, lds=305)
    assert relerr(S, ref) < 1e-6


@pytest.mark.parametrize("impl", [SIMT, TENSOR])
def test_spass_in_place(impl):
    S, ref, _ = _case(256, 130, 9, inplace=True, impl=impl)
    assert relerr(S, ref) < 1e-6


@pytest.mark.parametrize("impl", [SIMT, TENSOR])
def test_spass_large_ragged(impl):
    S, ref, _ = _case(4099, 1031, 20, seed=3, impl=impl)
    assert relerr(S, ref) < 1e-6


@pytest.mark.parametrize("m,n,r,ldm,lds,inplace", [
    (4099, 1031, 50, None, None, False),   # ragged tails
    (301, 97, 40, 303, 305, False),        # odd leading dimensions
    (256, 130, 64, None, None, True),      # in place
    (129, 33, 33, None, None, False)])
@pytest.mark.parametrize("impl", [SIMT, TENSOR])
def test_spass_high_rank(m, n, r, ldm, lds, inplace, impl):
    # ranks above 32 (the 20000 x 20000 rank-50 workload's range)
    S, ref, r = _case(m, n, r, ldm=ldm, lds=lds, seed=r, inplace=inplace,
                      impl=impl)
    err = np.abs(S - ref).max()
    bound = 4 * np.finfo(np.float32).eps * (10 * 4 + 2 * r * 4)
    assert err <= bound * np.sqrt(r), err
    assert relerr(S, ref) < 1e-6


def test_spass_tensor_refuses_what_it_cannot_tile():
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    M = torch.zeros((60, 200), device="cuda").t().contiguous().t()
    Lu = torch.zeros((60, 4), device="cuda").t().contiguous().t()
    Lv = torch.zeros((200, 4), device="cuda").t().contiguous().t()
    S = torch.empty_like(M)
    with pytest.raises(pk.PCPError, match="UNSUPPORTED"):
        pk.pcp_spass(M, Lu, Lv, S, impl=TENSOR)   # m < 128
    pk.pcp_spass(M, Lu, Lv, S, impl=0)            # the library's choice: SIMT
    torch.cuda.synchronize()


def test_spass_tensor_entrywise_bound_and_deterministic():
    # |S - S_exact| <= c 2^-21 (|Lu| |Lv|^T) + FP32 rounding of M - L, per entry
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    rng = np.random.default_rng(11)
    m, n, r = 2000, 1500, 50
    M = (rng.uniform(-10, 10, (m, n))).astype(np.float32)
    Lu = (rng.standard_normal((m, r)) / np.sqrt(r)).astype(np.float32)
    Lv = rng.standard_normal((n, r)).astype(np.float32)
    dM, dLu, dLv = to_dev_cm(M), to_dev_cm(Lu), to_dev_cm(Lv)
    dS1 = to_dev_cm(np.zeros((m, n), np.float32))
    dS2 = to_dev_cm(np.zeros((m, n), np.float32))
    pk.pcp_spass(dM, dLu, dLv, dS1, impl=TENSOR)
    pk.pcp_spass(dM, dLu, dLv, dS2, impl=TENSOR)
    torch.cuda.synchronize()
    S1, S2 = to_host(dS1), to_host(dS2)
    assert np.array_equal(S1, S2)
    L = Lu.astype(np.float64) @ Lv.astype(np.float64).T
    ref = M.astype(np.float64) - L
    B = np.abs(Lu.astype(np.float64)) @ np.abs(Lv.astype(np.float64)).T
    bound = 4 * 2.0 ** -21 * B + 2 * 2.0 ** -24 * (np.abs(M) + np.abs(L))
    assert np.all(np.abs(S1 - ref) <= bound)
