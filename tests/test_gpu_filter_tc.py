"""GPU parity of the tensor-core form of Algorithm 1 against the FP64 oracle.

The two products of every ADM iteration run as mma.sync with FP32
accumulation: split (three-pass) TF32 throughout for PCP_FP32_TENSOR, and
one-pass TF32 (PCP_TF32_REFINED) or one-pass BF16 (PCP_BF16_REFINED) for the
first lowp_iters iterations followed by split TF32 (the FP32 refinement).
All must give A z within
relative Frobenius error 1e-5 of the oracle (eps = 1e-10), for column and
row problems, ragged problem counts (not a multiple of the 16 problems per
CTA), lengths that are not a multiple of 8, and the large shapes the SIMT
kernel does not take (p up to 512, r up to 64).
"""
import numpy as np
import pytest

from oracle import l1filter
from tests.gpuhelp import relerr
from tests.test_gpu_filter import _problem, _run

pytestmark = pytest.mark.gpu

TOL = 1e-5
PCP_BF16_REFINED, PCP_TF32_REFINED, PCP_FP32_TENSOR = 1, 2, 4
PRECISIONS = [PCP_FP32_TENSOR, PCP_TF32_REFINED, PCP_BF16_REFINED]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("orientation", ["col", "row"])
@pytest.mark.parametrize("p,r,N", [(50, 5, 450), (200, 20, 100), (37, 3, 33),
                                   (200, 24, 65), (129, 17, 16), (64, 8, 1),
                                   (500, 50, 70), (300, 40, 33),
                                   (512, 64, 20)])
def test_tc_filter_matches_oracle(precision, orientation, p, r, N):
    A, X = _problem(2000 + p + N, p, r, N)
    Zg, it = _run(A, X, orientation, precision=precision)
    ref = l1filter.adm_l1(X, A)
    assert np.all(np.isfinite(Zg))
    assert relerr(A @ Zg, A @ ref.Z) < TOL
    colerr = np.linalg.norm(A @ (Zg - ref.Z), axis=0) / \
        np.maximum(np.linalg.norm(A @ ref.Z, axis=0), 1e-30)
    assert colerr.max() < 10 * TOL
    assert (it > 0).all()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_tc_zero_and_clean_columns(precision):
    rng = np.random.default_rng(7)
    p, r, N = 60, 4, 40
    A, _ = np.linalg.qr(rng.standard_normal((p, r)))
    A = A.astype(np.float32).astype(np.float64)
    X = (A @ rng.standard_normal((r, N))).astype(np.float32).astype(np.float64)
    X[:, 3] = 0.0
    X[:, 17] = 0.0
    Zg, it = _run(A, X, "col", precision=precision, lowp_iters=4)
    assert np.all(Zg[:, [3, 17]] == 0.0)
    assert it[3] == 0 and it[17] == 0
    mask = np.ones(N, bool)
    mask[[3, 17]] = False
    # uncorrupted columns: the least-squares z_1 is exact up to the split
    # products' rounding (~2^-21), so the stop test (3e-7 of ||x - e||_inf,
    # here ||x||_inf) is met on the first split-product iteration or the
    # one after
    # (after one-pass TF32 iterations, whose rounding leaves small nonzero
    # e entries, the refinement takes a few iterations more)
    first, extra = {PCP_FP32_TENSOR: (1, 2), PCP_TF32_REFINED: (5, 4),
                    PCP_BF16_REFINED: (5, 8)}[precision]
    assert (it[mask] >= first).all() and (it[mask] <= first + extra).all()
    assert relerr(Zg[:, mask], A.T @ X[:, mask]) < 1e-6


@pytest.mark.parametrize("precision", PRECISIONS)
def test_tc_rank_cap_scale_and_max_iter(precision):
    A, X = _problem(11, 80, 8, 70)
    sc = np.linspace(0.5, 2.0, 8)
    Zg, _ = _run(A, X, "row", rank=8, scale=sc, precision=precision)
    ref = l1filter.adm_l1(X, A)
    assert relerr(Zg / sc[:, None], ref.Z) < TOL
    # a rank-capped basis gives the same iterates as the basis of its first
    # columns (the regression on 5 of the 8 directions is a flat l1
    # problem, so it is compared with the same kernel, not the oracle)
    A5 = np.hstack([A[:, :5], np.zeros((80, 3))])
    Zc, _ = _run(A5, X, "col", rank=5, precision=precision)
    assert np.all(Zc[5:] == 0.0)
    Zr, _ = _run(A[:, :5], X, "col", precision=precision)
    np.testing.assert_allclose(Zc[:5], Zr, rtol=0,
                               atol=1e-6 * np.abs(Zr).max())
    A2, X2 = _problem(12, 100, 10, 40, dens=0.2)
    _, it = _run(A2, X2, "col", max_iter=2, precision=precision)
    assert (it == -2).all()


def test_tc_deterministic_and_matches_simt():
    A, X = _problem(13, 150, 12, 96)
    z1, _ = _run(A, X, "row", precision=PCP_FP32_TENSOR)
    z2, _ = _run(A, X, "row", precision=PCP_FP32_TENSOR)
    np.testing.assert_array_equal(z1, z2)
    zs, _ = _run(A, X, "row", precision=5)     # PCP_FP32_SIMT
    assert relerr(A @ z1, A @ zs) < TOL
    # PCP_FP32 runs whichever of the two kernels measured faster on this
    # shape class: its result is bit-identical to that kernel's
    zd, _ = _run(A, X, "row", precision=0)
    assert np.array_equal(zd, z1) or np.array_equal(zd, zs)
    zd2, _ = _run(A, X, "row", precision=0)
    np.testing.assert_array_equal(zd2, zd)


@pytest.mark.parametrize("precision", [PCP_BF16_REFINED, PCP_TF32_REFINED])
def test_error_before_and_after_refinement(precision, capsys):
    # the error of A z against the FP64 oracle after the lowp_iters one-pass
    # iterations alone (max_iter = lowp_iters stops the kernel there), beside
    # the FP32-accurate form stopped after as many iterations (the ADM's own
    # progress at that count) and the refined result at the FP32 stop test;
    # shapes of the 5000^2 r20 column filter (p = 200, r = 20, 10% outliers
    # of up to 100 against entries of a few units)
    A, X = _problem(31, 200, 20, 480, dens=0.1, mag=100.0)
    ref = l1filter.adm_l1(X, A)

    def err(Z):
        return relerr(A @ Z, A @ ref.Z)

    lowp = 12
    Zb, itb = _run(A, X, "col", precision=precision, lowp_iters=lowp,
                   max_iter=lowp)
    Zf, _ = _run(A, X, "col", precision=PCP_FP32_TENSOR, max_iter=lowp)
    Zr, itr = _run(A, X, "col", precision=precision, lowp_iters=lowp)
    eb, ef, er = err(Zb), err(Zf), err(Zr)
    with capsys.disabled():
        print(f"\nprecision {precision}: before refinement {eb:.3e} "
              f"(FP32 form at {lowp} iterations {ef:.3e}), after {er:.3e}, "
              f"iterations max {int(np.abs(itr).max())}")
    assert (itb == -lowp).all()        # stopped by max_iter, unrefined
    assert er < TOL and (itr > 0).all()
    assert eb > 100 * er

