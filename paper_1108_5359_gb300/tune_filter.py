"""Tuning run for the PCP_FP32 Algorithm 1 kernel choice (needs a GPU).

For every shape class both kernels take (p <= 64 / 128 / 256, r <= 8 / 16 /
24 / 32) this times adm_f32_kernel (PCP_FP32_SIMT) and adm_tc_kernel
(PCP_FP32_TENSOR) through pcp_l1_filter on the same synthetic problems
(4800 columns of a low-rank-plus-sparse matrix, entries at scattered rows,
like the column filter of a 5000 x 5000 solve), and writes
``csrc/filter_table.inc`` with the faster kernel per class.  The library
compiles the table in, so the choice is fixed per shape, not per process.

    python -m paper_1108_5359_gb300.tune_filter [--write]
"""
from __future__ import annotations

import argparse
import os
import statistics

import numpy as np

from . import _abi, build

P_CLASSES = (64, 128, 256)
R_CLASSES = (8, 16, 24, 32)
TABLE = os.path.join(build.CSRC, "filter_table.inc")


def _time_class(pk, torch, p, r, n_prob=4800, m=5000, reps=5, seed=0):
    rng = np.random.default_rng(seed + 7 * p + r)
    A, _ = np.linalg.qr(rng.standard_normal((p, r)))
    rows = np.sort(rng.choice(m, p, replace=False))
    Z = rng.standard_normal((r, n_prob)) * 5.0
    X = A @ Z
    mask = rng.random(X.shape) < 0.1
    X[mask] += rng.uniform(-100, 100, mask.sum())
    M = np.zeros((m, n_prob), dtype=np.float32, order="F")
    M[rows, :] = X
    dev = torch.device("cuda")
    dM = pk.colmajor(m, n_prob, device=dev)
    dM.copy_(torch.from_numpy(M))
    dA = pk.colmajor(p, r, device=dev)
    dA.copy_(torch.from_numpy(A.astype(np.float32)))
    pidx = torch.as_tensor(rows.astype(np.int32), device=dev)
    qidx = torch.arange(n_prob, dtype=torch.int32, device=dev)
    Zout = pk.colmajor(n_prob, r, device=dev)
    out = {}
    for name, prec in (("simt", _abi.PCP_FP32_SIMT),
                       ("tensor", _abi.PCP_FP32_TENSOR)):
        def run():
            pk.pcp_l1_filter(dM, pidx, 1, qidx, m, dA, r, Zout, n_prob, 3e-6,
                             1.5, precision=prec)
        for _ in range(2):
            run()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = statistics.median(ts)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true",
                    help="rewrite csrc/filter_table.inc")
    args = ap.parse_args()
    import torch
    import paper_1108_5359_gb300 as pk
    build.build()
    pk.load()
    table, lines = [], []
    for p in P_CLASSES:
        row = []
        for r in R_CLASSES:
            t = _time_class(pk, torch, p, r)
            k = _abi.PCP_KERNEL_SIMT if t["simt"] < t["tensor"] else \
                _abi.PCP_KERNEL_TENSOR
            row.append(k)
            lines.append(f"//   p={p:3d} r={r:2d}: SIMT {t['simt']:.3f} ms, "
                         f"tensor {t['tensor']:.3f} ms")
            print(lines[-1][5:], flush=True)
        table.append(row)
    gpu = torch.cuda.get_device_name()
    text = [
        "// Algorithm 1 kernel of PCP_FP32 per shape class: [p <= 64 / 128 / "
        "256]",
        "// [r <= 8 / 16 / 24 / 32]; 1 = adm_f32_kernel (FP32 SIMT), 2 = "
        "adm_tc_kernel",
        "// (split-TF32 tensor cores).  Written by "
        "`python -m paper_1108_5359_gb300.tune_filter --write`",
        f"// on {gpu}: median of 5 launches over 4800 problems per class "
        "(the faster",
        "// kernel is kept):",
        *lines,
        "static const int kFp32KernelTable[3][4] = {",
        *["    {" + ", ".join(str(k) for k in row) + "}," for row in table],
        "};",
    ]
    if args.write:
        with open(TABLE, "w") as f:
            f.write("\n".join(text) + "\n")
    print("\n".join(text))


if __name__ == "__main__":
    main()
