"""Seeded synthetic inputs shaped like the paper's experiments.

This module only builds inputs: it holds none of the method's arithmetic, so
both the FP64 oracle (through the tests) and the CUDA path consume exactly the
same arrays.  Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.

Data model (Section 1, model of M = L0 + S0; Section 4.1 generator):
  * L0 = X Y^T with X (m x r), Y (n x r) i.i.d. Gaussian;
  * S0 has a support chosen uniformly at random, its nonzeros i.i.d. uniform
    in [lo, hi].

Matrices are returned column-major (Fortran order), the layout the library's
C ABI takes (leading dimension >= m).  The observation handed to the GPU is
``M32 = M.astype(float32)``; the oracle is fed ``M32.astype(float64)`` so that
both sides see bit-identical inputs.

The seed index sets I_s, J_s (Algorithm 2, step 1: a random submatrix) are
drawn here too and passed to both sides as inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem",
    "lowrank_plus_sparse",
    "seed_indices",
    "make_config",
    "CONFIGS",
    "lowrank_factors",
    "seed_orders",
    "uneven_instances",
    "video_like",
    "checkerboard",
    "sparse_magnitude",
]


@dataclasses.dataclass
class Problem:
    """One PCP instance M = L0 + S0 with its seed index sets."""

    M: np.ndarray          # m x n, float64, column-major
    L0: np.ndarray | None  # ground truth (None when too large to keep)
    S0: np.ndarray | None
    r: int
    rows: np.ndarray       # I_s, sorted int64
    cols: np.ndarray       # J_s, sorted int64
    name: str = ""

    @property
    def m(self) -> int:
        return self.M.shape[0]

    @property
    def n(self) -> int:
        return self.M.shape[1]

    def m32(self) -> np.ndarray:
        return np.asfortranarray(self.M.astype(np.float32))


def _flat(seed):
    if isinstance(seed, (tuple, list)):
        out = []
        for s in seed:
            out.extend(_flat(s))
        return out
    return [int(seed)]


def _rng(seed) -> np.random.Generator:
    """PCG64 generator; ``seed`` is an int or a (nested) tuple of ints."""
    return np.random.Generator(np.random.PCG64(_flat(seed)))


def _sparse_support(rng, m, n, density, exact=None):
    """Boolean mask of a uniformly random support.

    With ``exact`` (default: when m*n <= 5e7) exactly round(density*m*n)
    positions are chosen without replacement, as the paper's generator does
    (p nonzeros); otherwise each entry is kept independently with the given
    probability (same distribution of positions, binomial count).
    """
    total = m * n
    if exact is None:
        exact = total <= 50_000_000
    mask = np.zeros(total, dtype=bool)
    if exact:
        p = int(round(density * total))
        if p > 0:
            mask[rng.choice(total, size=p, replace=False)] = True
    else:
        mask = rng.random(total) < density
    return mask.reshape((m, n), order="F")


def lowrank_plus_sparse(m, n, r, density, lo, hi, seed=0, factor_std=1.0,
                        keep_truth=True, dtype=np.float64):
    """M = X Y^T + S0 (Section 4.1 generator).

    X, Y have i.i.d. N(0, factor_std^2) entries; S0's support is uniform with
    the given density and its values are i.i.d. U[lo, hi].
    """
    rng = _rng(seed)
    X = rng.standard_normal((m, r)) * factor_std
    Y = rng.standard_normal((n, r)) * factor_std
    L0 = np.asfortranarray(X @ Y.T)
    mask = _sparse_support(rng, m, n, density)
    vals = rng.uniform(lo, hi, size=int(mask.sum()))
    S0 = np.zeros((m, n), order="F")
    S0[mask] = vals  # boolean assignment fills in the mask's (C-)order
    # sum in FP64, then round once to the storage type
    M = np.asfortranarray((L0 + S0).astype(dtype, copy=False))
    if not keep_truth:
        return M, None, None
    return M, L0.astype(dtype, copy=False), S0.astype(dtype, copy=False)


def lowrank_factors(m, n, r, seed=0, factor_std=1.0):
    """The X (m x r) and Y (n x r) that lowrank_plus_sparse draws for the
    same seed (L0 = X Y^T), for checking sampled entries of a large L0."""
    rng = _rng(seed)
    X = rng.standard_normal((m, r)) * factor_std
    Y = rng.standard_normal((n, r)) * factor_std
    return X, Y


def seed_orders(m, n, rows, cols, seed=0):
    """Row and column sampling orders whose first entries are the given
    seed sets (then the remaining indices in random order), for seeds that
    may grow by prefixes (Section 3.5)."""
    rng = _rng((seed, 0x0DE2))
    out = []
    for size, first in ((m, rows), (n, cols)):
        first = np.asarray(first, dtype=np.int64)
        rest = np.setdiff1d(np.arange(size), first)
        out.append(np.concatenate([rng.permutation(first),
                                   rng.permutation(rest)]))
    return out[0], out[1]


def seed_indices(m, n, mp, np_, seed=0):
    """Uniform random I_s (|I_s| = mp) and J_s (|J_s| = np_), sorted.

    Algorithm 2 step 1 samples the seed submatrix at random; the sets need not
    be contiguous (Section 1.1 footnote).  Drawn without replacement.
    """
    rng = _rng((seed, 0x5EED))
    rows = np.sort(rng.choice(m, size=mp, replace=False)).astype(np.int64)
    cols = np.sort(rng.choice(n, size=np_, replace=False)).astype(np.int64)
    return rows, cols


# Workload shapes.  "s" is the oversampling rate s_r = s_c (Section 3.1
# chooses 10), so the seed is (s r) x (s r).
CONFIGS = {
    # 500^2, rank 5, 5% support in [-50, 50], seed 50 x 50
    "c1_500_r5": dict(m=500, n=500, r=5, density=0.05, lo=-50.0, hi=50.0,
                      factor_std=1.0, s=10),
    # 5000^2, rank 20, 10% support in [-100, 100], seed 200 x 200
    "c2_5000_r20": dict(m=5000, n=5000, r=20, density=0.10, lo=-100.0,
                        hi=100.0, factor_std=1.0, s=10),
    # 20000^2, rank 50, X,Y ~ N(0, 1/r), 10% support in [-10, 10], seed 500^2
    "c3_20000_r50": dict(m=20000, n=20000, r=50, density=0.10, lo=-10.0,
                         hi=10.0, factor_std=1.0 / math.sqrt(50.0), s=10),
    # Table 1 shapes (rho_r = rho_s = 0.01, values in [-500, 500])
    "t1_2000_r20": dict(m=2000, n=2000, r=20, density=0.01, lo=-500.0,
                        hi=500.0, factor_std=1.0, s=10),
}


def make_config(name, seed=0, keep_truth=True, dtype=np.float64, **override):
    """Build the Problem for a named workload shape (optionally overridden)."""
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    m, n, r = cfg["m"], cfg["n"], cfg["r"]
    M, L0, S0 = lowrank_plus_sparse(
        m, n, r, cfg["density"], cfg["lo"], cfg["hi"], seed=seed,
        factor_std=cfg["factor_std"], keep_truth=keep_truth, dtype=dtype)
    s = cfg["s"]
    rows, cols = seed_indices(m, n, s * r, s * r, seed=seed)
    return Problem(M=M, L0=L0, S0=S0, r=r, rows=rows, cols=cols, name=name)


def uneven_instances(count=256, seed=0, m_range=(300, 4000),
                     n_range=(200, 3000), r_max=30, density_range=(0.02, 0.15),
                     lo=-50.0, hi=50.0, s=10, keep_truth=True,
                     dtype=np.float64, indices=None):
    """Many instances of different sizes (batched workload).

    m ~ U[m_range], n ~ U[n_range], r ~ U[3, min(r_max, floor(min(m, n)/20))]
    (so that the 10r x 10r seed stays within half of each dimension, the size
    limit of the target-rank test in Section 3.5), density ~ U[density_range].
    ``indices`` builds only those instances (the sizes of all are drawn in
    order, so instance i is the same whichever subset is built).
    """
    rng = _rng((seed, 0xBA7C))
    want = None if indices is None else set(int(i) for i in indices)
    out = []
    for i in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        rmax = max(3, min(r_max, min(m, n) // 20))
        r = int(rng.integers(3, rmax + 1))
        dens = float(rng.uniform(*density_range))
        if want is not None and i not in want:
            continue
        M, L0, S0 = lowrank_plus_sparse(m, n, r, dens, lo, hi,
                                        seed=(seed, i, 1),
                                        keep_truth=keep_truth, dtype=dtype)
        rows, cols = seed_indices(m, n, s * r, s * r, seed=(seed, i, 2))
        out.append(Problem(M=M, L0=L0, S0=S0, r=r, rows=rows, cols=cols,
                           name=f"uneven{i}"))
    return out


def _blur1d(a, sigma, axis):
    """Separable Gaussian blur along one axis (zero padded)."""
    rad = int(math.ceil(3 * sigma))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    n = a.shape[axis]
    return np.apply_along_axis(
        lambda v: np.convolve(v, k, mode="full")[rad:rad + n], axis, a)


def video_like(n_frames, height=240, width=320, r=None, seed=0,
               cover_range=(0.05, 0.15), fg_lo=0.2, fg_hi=1.0, blur_px=8.0):
    """Background-modelling shaped instance (Section 4.3 shape).

    Each column is one flattened frame (m = height*width).  L0 = sum_k a_k b_k^T
    with a_k a blurred Gaussian image scaled to [0, 1] and b_k a smooth
    temporal curve; S0 per frame is a set of random axis-aligned rectangles
    whose union covers a fraction f ~ U[cover_range] of the frame, values
    U[fg_lo, fg_hi] (the last rectangle wins on overlap).
    """
    rng = _rng((seed, 0x71DE0))
    m = height * width
    if r is None:
        r = int(rng.integers(1, 6))
    A = np.empty((m, r))
    B = np.empty((n_frames, r))
    for k in range(r):
        img = rng.standard_normal((height, width))
        img = _blur1d(_blur1d(img, blur_px, 0), blur_px, 1)
        img = (img - img.min()) / max(img.max() - img.min(), 1e-12)
        A[:, k] = img.reshape(-1, order="F")
        curve = np.cumsum(rng.standard_normal(n_frames))
        curve = _blur1d(curve, 5.0, 0)
        B[:, k] = 1.0 + 0.1 * curve / max(np.abs(curve).max(), 1e-12)
    L0 = np.asfortranarray(A @ B.T)
    S0 = np.zeros((m, n_frames), order="F")
    # rectangle sides in [8, side/3) px (narrower bounds on tiny frames)
    hlo = max(2, min(8, height // 6))
    hhi = max(hlo + 1, height // 3)
    wlo = max(2, min(8, width // 6))
    whi = max(wlo + 1, width // 3)
    for j in range(n_frames):
        frame = np.zeros((height, width))
        mask = np.zeros((height, width), dtype=bool)
        target = rng.uniform(*cover_range)
        while mask.mean() < target:
            h = int(rng.integers(hlo, hhi))
            w = int(rng.integers(wlo, whi))
            y0 = int(rng.integers(0, height - h))
            x0 = int(rng.integers(0, width - w))
            frame[y0:y0 + h, x0:x0 + w] = rng.uniform(fg_lo, fg_hi)
            mask[y0:y0 + h, x0:x0 + w] = True
        S0[:, j] = frame.reshape(-1, order="F")
    M = np.asfortranarray(L0 + S0)
    s = 10
    mp = max(20, s * r)
    rows, cols = seed_indices(m, n_frames, mp, max(20, s * r),
                              seed=(seed, 0x71DE1))
    return Problem(M=M, L0=L0, S0=S0, r=r, rows=rows, cols=cols,
                   name="video_like")


def checkerboard(m, square=None, density=0.10, seed=0, seed_size=60):
    """Rank-2 checkerboard corrupted by impulsive noise (Section 4.1.2 shape).

    Entries are 0/1 squares (``square`` pixels wide, default m // 8); 10% of
    entries (uniform support) are replaced by the opposite colour (impulsive
    noise), i.e. S0 = flipped - L0.  The section gives no seed size: at this
    corruption a 20 x 20 seed (10 r) does not recover the seed's own low-rank
    part, a 60 x 60 one (30 r) does, so ``seed_size`` defaults to 60.
    """
    rng = _rng((seed, 0xC4EC))
    if square is None:
        square = max(1, m // 8)
    idx = (np.arange(m) // square) % 2
    L0 = np.asfortranarray((idx[:, None] ^ idx[None, :]).astype(np.float64))
    mask = _sparse_support(rng, m, m, density)
    S0 = np.zeros((m, m), order="F")
    S0[mask] = 1.0 - 2.0 * L0[mask]
    M = np.asfortranarray(L0 + S0)
    rows, cols = seed_indices(m, m, seed_size, seed_size, seed=seed)
    return Problem(M=M, L0=L0, S0=S0, r=2, rows=rows, cols=cols,
                   name="checkerboard")


def sparse_magnitude(sigma, m=1000, seed=0, s=10):
    """M = L0 + sigma S0 with the Section 4.1 generator (Section 4.1.2 sweep).

    m x m, r = 0.01 m, support ratio 0.01, S0's values U[-500, 500] before the
    scale sigma (the sweep runs sigma from 1 to 10); the seed is (s r)^2.
    """
    r = max(1, int(round(0.01 * m)))
    M, L0, S0 = lowrank_plus_sparse(m, m, r, 0.01, -500.0, 500.0, seed=seed)
    S0 = np.asfortranarray(sigma * S0)
    M = np.asfortranarray(L0 + S0)
    rows, cols = seed_indices(m, m, s * r, s * r, seed=seed)
    return Problem(M=M, L0=L0, S0=S0, r=r, rows=rows, cols=cols,
                   name=f"sparse_magnitude_{sigma:g}")
