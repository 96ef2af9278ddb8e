"""GPU parity on the background-modelling shape (Section 4.3).

A 76800 x 300 matrix of flattened 320 x 240 frames: a smooth background of
rank 3 and a foreground of random rectangles covering 5-15% of every frame
(values U[0.2, 1]), the stand-in for the paper's videos.  The corruption is
structured, not the uniform support the recovery theory assumes: the first
30 x 30 seed's recovered L^s has raw rank 5 (foreground leakage at 3e-5 and
3e-6 of sigma_1), so Eq. rank_test fails and, with Section 3.5's rule, the
seed grows to 50 x 50 on both sides.  Neither side recovers L0 exactly
(~8e-4 relative).

What is checked, and at which level:
  * Algorithm 1 alone (pcp_l1_filter) on the video shape's 250 column and
    76750 row problems, with the oracle's own seed factors as A: the
    FP32-accurate forms match the oracle's Q~ and P~ within 1e-5 (measured
    ~1e-6); the one-pass BF16 / TF32 forms with FP32 refinement are stated
    per result (measured 1.2e-4 / 1.5e-5 on this input, whose l1 problems
    are flat near their minimisers) and bounded by 1e-3.
  * The whole solve (seed growth, seed PCP, filters, S pass) against the
    oracle on the same grown seed: bounded by 2e-4 on L in the FP32 form
    (measured 6e-5) and by 1e-3 in the refined forms.
    The gap to 1e-5 is the seed's: this seed's spectrum spans
    sigma_4 / sigma_1 ~ 4e-5, so its Rayleigh-Ritz matrix spans ~1e-9,
    below the resolution of the FP32 k x k eigen-solve inside the device
    ALM; the seed's L^s differs from the oracle's by ~5e-5 (measured, and
    independent of the subspace size).  The uniform-corruption workloads
    (spectra within two decades) hold 1e-5 end to end (test_gpu_solve.py).
"""
import numpy as np
import pytest

from oracle import l1filter
from paper_1108_5359_gb300 import synth
from tests.gpuhelp import build_and_load, idx_dev, relerr, to_dev_cm, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5
FP32_FORMS = [0, 4, 5]   # PCP_FP32 (table), PCP_FP32_TENSOR, PCP_FP32_SIMT
REFINED_FORMS = [1, 2]   # PCP_BF16_REFINED, PCP_TF32_REFINED


@pytest.fixture(scope="module")
def video():
    P = synth.video_like(300, seed=1)
    ro, co = synth.seed_orders(P.m, P.n, P.rows, P.cols, seed=1)
    M32 = P.M.astype(np.float32)
    rows, cols = np.sort(ro[:50]), np.sort(co[:50])   # the grown seed
    ref = l1filter.l1_filter_pcp(M32.astype(np.float64), rows, cols, r=P.r)
    assert ref.rank_ok and ref.rank == P.r
    return P, M32, ro, co, rows, cols, ref


@pytest.mark.parametrize("precision", FP32_FORMS + REFINED_FORMS)
def test_video_filters_with_the_oracle_seed(video, precision):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P, M32, _, _, rows, cols, ref = video
    r = P.r
    dM = to_dev_cm(M32)
    rbar = np.setdiff1d(np.arange(P.m), rows)
    cbar = np.setdiff1d(np.arange(P.n), cols)
    Zc, Zr = pk.colmajor(P.n, r), pk.colmajor(P.m, r)
    pk.pcp_l1_filter(dM, idx_dev(rows), 1, idx_dev(cbar), dM.stride(1),
                     to_dev_cm(ref.U.astype(np.float32)), r, Zc, P.n, 3e-6,
                     1.5, precision=precision)
    pk.pcp_l1_filter(dM, idx_dev(cols), dM.stride(1), idx_dev(rbar), 1,
                     to_dev_cm(ref.V.astype(np.float32)), r, Zr, P.m, 3e-6,
                     1.5, precision=precision)
    torch.cuda.synchronize()
    ec = relerr(to_host(Zc)[cbar], ref.Qt.T)
    er = relerr(to_host(Zr)[rbar], ref.Pt.T)
    print(f"\nvideo Algorithm 1, precision {precision}: column problems "
          f"{ec:.2e}, row problems {er:.2e} against the oracle")
    bound = TOL if precision in FP32_FORMS else 1e-3
    assert ec < bound and er < bound


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_video_whole_solve(video, precision):
    import torch
    import paper_1108_5359_gb300 as pk
    build_and_load()
    P, M32, ro, co, rows0, cols0, ref = video
    dM = to_dev_cm(M32)
    p = pk.pcp_params_default(P.m, P.n, P.r)
    p.precision = precision
    p.grow_seed = 1
    plan = pk.Plan(p, row_order=ro, col_order=co)
    Lu, Lv = pk.colmajor(P.m, P.r), pk.colmajor(P.n, P.r)
    S = pk.colmajor(P.m, P.n)
    st, info, rows, cols = pk.pcp_l1filter_solve(plan, dM, Lu, Lv, S,
                                                 raise_on_error=False)
    torch.cuda.synchronize()
    plan.close()
    assert st == 0, info.as_dict()
    assert info.seed_m == info.seed_n == 50       # grown from 30 x 30
    np.testing.assert_array_equal(rows, rows0)
    np.testing.assert_array_equal(cols, cols0)
    assert info.rank == ref.rank == P.r
    L = to_host(Lu) @ to_host(Lv).T
    e_L, e_S = relerr(L, ref.L), relerr(to_host(S), ref.S)
    e0 = relerr(L, P.L0)
    print(f"\nvideo whole solve, precision {precision}: L vs oracle "
          f"{e_L:.2e}, S vs oracle {e_S:.2e}, L vs L0 {e0:.2e} (oracle "
          f"{relerr(ref.L, P.L0):.2e})")
    assert e_L < (2e-4 if precision == 0 else 1e-3)
    assert e0 < 1e-2
