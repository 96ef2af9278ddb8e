"""GB300-native l1 filtering for Principal Component Pursuit (arXiv 1108.5359).

The work runs in the CUDA library ``libpcpl1f.so`` (C ABI in
``include/pcp_l1f.h``); this module only marshals torch tensors (device
memory, streams) into its entry points, under the same names.  There is no
CPU fallback: every call fails if the library or a GPU is missing.

Matrix convention: column-major.  A torch tensor ``X`` of shape (rows, cols)
is passed as (pointer, leading dimension) and must have ``X.stride(0) == 1``;
``colmajor(rows, cols)`` allocates one.
"""
from __future__ import annotations

import ctypes as C

from . import _abi
from ._abi import (PCPError, PCPInfo, PCPParams, PCPProblem,
                   PCP_BF16_REFINED, PCP_ERR_BUSY, PCP_FP32, PCP_FP32_SIMT,
                   PCP_FP32_TENSOR, PCP_OK, PCP_TF32_REFINED,
                   PCP_SPASS_AUTO, PCP_SPASS_SIMT, PCP_SPASS_TENSOR, check,
                   load)

__all__ = [
    "PCPError", "PCPInfo", "PCPParams", "PCP_FP32", "PCP_BF16_REFINED",
    "PCP_TF32_REFINED", "PCP_FP32_TENSOR", "PCP_FP32_SIMT",
    "colmajor", "pcp_params_default", "pcp_l1filter_plan",
    "pcp_l1filter_solve", "pcp_l1filter_solve_host", "pcp_plan_destroy",
    "pcp_plan_graph_launches",
    "pcp_gather_seed",
    "pcp_seed_workspace_bytes", "pcp_seed_pcp", "pcp_seed_pcp_static",
    "pcp_l1_filter", "pcp_l1_filter_kernel",
    "pcp_assemble_factors", "pcp_spass", "PCP_SPASS_AUTO", "PCP_SPASS_SIMT",
    "PCP_SPASS_TENSOR", "pcp_plan_seed_trace", "Plan",
    "solve", "load", "SEED_PHASES", "PCPProblem", "problem",
    "pcp_l1filter_batch", "BatchPlan", "pcp_l1filter_batch_plan",
    "pcp_l1filter_batch_run", "pcp_batch_plan_destroy", "Server", "pcp_serve_create", "pcp_serve_submit",
    "pcp_serve_poll", "pcp_serve_wait", "pcp_serve_stop", "pcp_serve_destroy",
]


def _torch():
    import torch
    return torch


def colmajor(rows, cols, dtype=None, device="cuda", fill=None):
    """Column-major (Fortran-order) tensor of shape (rows, cols)."""
    torch = _torch()
    dtype = dtype or torch.float32
    t = torch.empty((cols, rows), dtype=dtype, device=device).t()
    if fill is not None:
        t.fill_(fill)
    return t


def _cm(t, name):
    """(pointer, leading dimension) of a column-major CUDA tensor."""
    if t is None:
        return None, 0
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() == 1:
        return t.data_ptr(), max(1, t.shape[0])
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return t.data_ptr(), max(t.stride(1), t.shape[0], 1)


def _cm_host(t, name):
    """(pointer, leading dimension) of a column-major CPU tensor (pinned for
    overlapped copies)."""
    if t is None:
        return None, 0
    if t.is_cuda:
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dim() == 2 and t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    if t.dim() == 1:
        return t.data_ptr(), max(1, t.shape[0])
    return t.data_ptr(), max(t.stride(1), t.shape[0], 1)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# --------------------------------------------------------------------------
# thin wrappers, one per C entry point
# --------------------------------------------------------------------------

def pcp_params_default(m, n, r) -> PCPParams:
    p = PCPParams()
    check(load().pcp_params_default(C.byref(p), m, n, r), "pcp_params_default")
    return p


def _set_index_arrays(params, keep, seed_rows, seed_cols, row_order,
                      col_order):
    """Point params' optional host index arrays at int64 copies kept alive
    in ``keep``.  A seed index set also sets the seed's size (seed_m /
    seed_n) to its length; a size already set to another value is an
    error (the library would read only that many entries)."""
    import numpy as np
    for name, v, size in (("seed_rows", seed_rows, "seed_m"),
                          ("seed_cols", seed_cols, "seed_n"),
                          ("row_order", row_order, None),
                          ("col_order", col_order, None)):
        if v is not None:
            a = np.ascontiguousarray(v, dtype=np.int64).ravel()
            if size is not None:
                have = getattr(params, size)
                if have and have != a.size:
                    raise ValueError(f"{name} has {a.size} entries but "
                                     f"params.{size} = {have}")
                setattr(params, size, a.size)
            keep.append(a)
            setattr(params, name, a.ctypes.data_as(C.POINTER(C.c_int64)))


class Plan:
    """Owns a pcp_plan (device workspace) and the index arrays it points to."""

    def __init__(self, params: PCPParams, seed_rows=None, seed_cols=None,
                 row_order=None, col_order=None):
        self._keep = []
        params = PCPParams.from_buffer_copy(params)
        _set_index_arrays(params, self._keep, seed_rows, seed_cols,
                          row_order, col_order)
        self.params = params
        self.handle = C.c_void_p()
        check(load().pcp_l1filter_plan(C.byref(params), C.byref(self.handle)),
              "pcp_l1filter_plan")
        self.m, self.n, self.r = params.m, params.n, params.r
        self.mp = params.seed_m or int(round(params.s_r * params.r))
        self.np = params.seed_n or int(round(params.s_c * params.r))
        self.grow = bool(params.grow_seed)

    def close(self):
        if self.handle:
            load().pcp_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcp_l1filter_plan(params: PCPParams, seed_rows=None, seed_cols=None,
                      row_order=None, col_order=None):
    return Plan(params, seed_rows, seed_cols, row_order, col_order)


def pcp_plan_destroy(plan: Plan):
    plan.close()


def pcp_l1filter_solve(plan: Plan, M, Lu, Lv, S=None, info=True,
                       stream=None, raise_on_error=True):
    """Algorithm 2 on M into (Lu, Lv, S); returns (status, info, rows, cols)."""
    import numpy as np
    pM, ldm = _cm(M, "M")
    pLu, _ = _cm(Lu, "Lu")
    pLv, _ = _cm(Lv, "Lv")
    pS, lds = _cm(S, "S")
    # a grown seed (Section 3.5) can reach min(512, m/2) x min(512, n/2)
    cap_r = max(plan.mp, min(512, plan.m // 2)) if plan.grow else plan.mp
    cap_c = max(plan.np, min(512, plan.n // 2)) if plan.grow else plan.np
    rows = np.zeros(cap_r, dtype=np.int64)
    cols = np.zeros(cap_c, dtype=np.int64)
    inf = PCPInfo() if info else None
    st = load().pcp_l1filter_solve(
        plan.handle, pM, ldm, pLu, pLv, pS, lds if S is not None else plan.m,
        rows.ctypes.data_as(C.POINTER(C.c_int64)),
        cols.ctypes.data_as(C.POINTER(C.c_int64)),
        C.byref(inf) if inf is not None else None, _stream(stream))
    if inf is not None and inf.seed_m:
        rows, cols = rows[:inf.seed_m], cols[:inf.seed_n]
    else:
        rows, cols = rows[:plan.mp], cols[:plan.np]
    if raise_on_error and st not in (PCP_OK,):
        check(st, "pcp_l1filter_solve")
    return st, inf, rows, cols


def pcp_plan_graph_launches(plan: Plan) -> int:
    """CUDA-graph replays of asynchronous solves on this plan (-1: off)."""
    return int(load().pcp_plan_graph_launches(plan.handle))


def pcp_l1filter_solve_host(plan: Plan, M, Lu, Lv, S=None, info=True,
                            stream=None, raise_on_error=True):
    """Algorithm 2 on a host M (column-major CPU tensor, pinned for overlap)
    into host (Lu, Lv, S), copies overlapped with compute; returns
    (status, info).  Without info, synchronise `stream` before reading."""
    pM, ldm = _cm_host(M, "M")
    pLu, _ = _cm_host(Lu, "Lu")
    pLv, _ = _cm_host(Lv, "Lv")
    pS, lds = _cm_host(S, "S")
    inf = PCPInfo() if info else None
    st = load().pcp_l1filter_solve_host(
        plan.handle, pM, ldm, pLu, pLv, pS, lds if S is not None else plan.m,
        C.byref(inf) if inf is not None else None, _stream(stream))
    if raise_on_error and st not in (PCP_OK,):
        check(st, "pcp_l1filter_solve_host")
    return st, inf


class _Problem:
    """A pcp_problem plus the host arrays its seed index pointers refer to."""

    def __init__(self, params, M, Lu, Lv, S=None, seed_rows=None,
                 seed_cols=None, row_order=None, col_order=None):
        self._keep = [M, Lu, Lv, S]
        p = PCPParams.from_buffer_copy(params)
        _set_index_arrays(p, self._keep, seed_rows, seed_cols, row_order,
                          col_order)
        pM, ldm = _cm(M, "M")
        pLu, _ = _cm(Lu, "Lu")
        pLv, _ = _cm(Lv, "Lv")
        pS, lds = _cm(S, "S")
        self.c = PCPProblem(p, pM, ldm, pLu, pLv, pS,
                            lds if S is not None else p.m)


def problem(params, M, Lu, Lv, S=None, seed_rows=None, seed_cols=None,
            row_order=None, col_order=None):
    """One instance for pcp_l1filter_batch / pcp_serve_submit (tensors as
    for pcp_l1filter_solve; Lu must be m x r and Lv n x r with ld m / n)."""
    return _Problem(params, M, Lu, Lv, S, seed_rows, seed_cols, row_order,
                    col_order)


def pcp_l1filter_batch(problems, info=True, stream=None,
                       raise_on_error=True):
    """Batched Algorithm 2; returns (status, [PCPInfo per instance] or None)."""
    n = len(problems)
    arr = (PCPProblem * max(n, 1))(*[q.c for q in problems])
    infos = (PCPInfo * max(n, 1))() if info else None
    st = load().pcp_l1filter_batch(n, arr, infos, _stream(stream))
    if raise_on_error and st != PCP_OK:
        check(st, "pcp_l1filter_batch")
    return st, (list(infos)[:n] if infos is not None else None)


class BatchPlan:
    """Owns a pcp_batch_plan (workspace + captured graph of a batch) and the
    problems' tensors it reads and writes on every run."""

    def __init__(self, problems, stream=None):
        n = len(problems)
        self._problems = list(problems)
        arr = (PCPProblem * max(n, 1))(*[q.c for q in problems])
        self.count = n
        self.handle = C.c_void_p()
        check(load().pcp_l1filter_batch_plan(n, arr, _stream(stream),
                                             C.byref(self.handle)),
              "pcp_l1filter_batch_plan")

    def run(self, info=True, stream=None, raise_on_error=True):
        """Replay the batch; returns (status, [PCPInfo] or None)."""
        infos = (PCPInfo * max(self.count, 1))() if info else None
        st = load().pcp_l1filter_batch_run(self.handle, infos,
                                           _stream(stream))
        if raise_on_error and st != PCP_OK:
            check(st, "pcp_l1filter_batch_run")
        return st, (list(infos)[:self.count] if infos is not None else None)

    def close(self):
        if self.handle:
            load().pcp_batch_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcp_l1filter_batch_plan(problems, stream=None):
    return BatchPlan(problems, stream)


def pcp_l1filter_batch_run(plan, info=True, stream=None, raise_on_error=True):
    return plan.run(info, stream, raise_on_error)


def pcp_batch_plan_destroy(plan):
    plan.close()


class Server:
    """Owns a pcp_server; keeps each request's tensors alive until polled."""

    def __init__(self, hbm_budget_bytes, max_slots=256, streams=4):
        self.handle = C.c_void_p()
        check(load().pcp_serve_create(int(hbm_budget_bytes), int(max_slots),
                                      int(streams), C.byref(self.handle)),
              "pcp_serve_create")
        self._live = {}

    def submit(self, prob):
        t = C.c_uint64()
        check(load().pcp_serve_submit(self.handle, C.byref(prob.c),
                                      C.byref(t)), "pcp_serve_submit")
        self._live[t.value] = prob
        return t.value

    def poll(self, ticket):
        """(status, PCPInfo) or (PCP_ERR_BUSY, None) while pending."""
        inf = PCPInfo()
        st = load().pcp_serve_poll(self.handle, ticket, C.byref(inf))
        if st == PCP_ERR_BUSY:
            return st, None
        self._live.pop(ticket, None)
        return st, inf

    def wait(self, ticket):
        inf = PCPInfo()
        st = load().pcp_serve_wait(self.handle, ticket, C.byref(inf))
        self._live.pop(ticket, None)
        return st, inf

    def stop(self):
        if self.handle:
            check(load().pcp_serve_stop(self.handle), "pcp_serve_stop")

    def close(self):
        if self.handle:
            load().pcp_serve_destroy(self.handle)
            self.handle = C.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcp_serve_create(hbm_budget_bytes, max_slots=256, streams=4):
    return Server(hbm_budget_bytes, max_slots, streams)


def pcp_serve_submit(server, prob):
    return server.submit(prob)


def pcp_serve_poll(server, ticket):
    return server.poll(ticket)


def pcp_serve_wait(server, ticket):
    return server.wait(ticket)


def pcp_serve_stop(server):
    server.stop()


def pcp_serve_destroy(server):
    server.close()


def pcp_gather_seed(M, d_rows, d_cols, Ms, stream=None):
    pM, ldm = _cm(M, "M")
    check(load().pcp_gather_seed(pM, ldm, _ptr(d_rows), d_rows.numel(),
                                 _ptr(d_cols), d_cols.numel(), _ptr(Ms),
                                 _stream(stream)), "pcp_gather_seed")


def pcp_seed_workspace_bytes(mp, np_, kmax):
    return int(load().pcp_seed_workspace_bytes(mp, np_, kmax))


def pcp_seed_pcp(D, lam, tol, rho, mu_scale, mu_max_ratio, max_iter, k0, kmax,
                 rank_cut, r_cap, work, U, Sigma, V, stream=None,
                 raise_on_error=True):
    mp, np_ = D.shape
    rank = C.c_int32()
    iters = C.c_int32()
    resid = C.c_double()
    pD, ldd = _cm(D, "D")
    if ldd != mp:
        raise ValueError("D must be packed (ld == rows)")
    st = load().pcp_seed_pcp(pD, mp, np_, lam, tol, rho, mu_scale,
                             mu_max_ratio, max_iter, k0, kmax, rank_cut, r_cap,
                             _ptr(work), _ptr(U), _ptr(Sigma), _ptr(V),
                             C.byref(rank), C.byref(iters), C.byref(resid),
                             _stream(stream))
    if raise_on_error:
        check(st, "pcp_seed_pcp")
    return st, rank.value, iters.value, resid.value


def pcp_seed_pcp_static(D, lam, tol, rho, mu_scale, mu_max_ratio, max_iter,
                        k0, kmax, rank_cut, r_cap, U, Sigma, V, stream=None,
                        raise_on_error=True):
    """pcp_seed_pcp without a workspace argument (library-owned scratch)."""
    mp, np_ = D.shape
    rank = C.c_int32()
    iters = C.c_int32()
    resid = C.c_double()
    pD, ldd = _cm(D, "D")
    if ldd != mp:
        raise ValueError("D must be packed (ld == rows)")
    st = load().pcp_seed_pcp_static(pD, mp, np_, lam, tol, rho, mu_scale,
                                    mu_max_ratio, max_iter, k0, kmax,
                                    rank_cut, r_cap, _ptr(U), _ptr(Sigma),
                                    _ptr(V), C.byref(rank), C.byref(iters),
                                    C.byref(resid), _stream(stream))
    if raise_on_error:
        check(st, "pcp_seed_pcp_static")
    return st, rank.value, iters.value, resid.value


def pcp_plan_seed_trace(plan, cap=4096, stream=None):
    """(timestamp_ns, phase) records of the plan's last seed solve."""
    import numpy as np
    buf = np.zeros(2 * cap, dtype=np.uint64)
    n = load().pcp_plan_seed_trace(plan.handle,
                                   buf.ctypes.data_as(C.POINTER(C.c_uint64)),
                                   cap, _stream(stream))
    if n < 0:
        raise PCPError(n, "pcp_plan_seed_trace failed")
    return buf[:2 * n].reshape(n, 2)


SEED_PHASES = {1: "prologue", 2: "T=G^T Omega", 3: "gram(T)", 4: "cholqr(T)",
               5: "P=G Psi", 6: "gram(P)", 7: "power orth", 8: "jacobi",
               9: "rotate", 10: "alm start", 11: "alm update",
               12: "jacobi setup", 13: "refine gram(Pt)",
               14: "refine apply", 15: "final FP64 SVD"}


def pcp_l1_filter(M, d_pidx, sp, d_qidx, sq, A, r, Z, ldz, eps, rho,
                  beta0_scale=1.0, beta_bar_ratio=1e10, max_iter=500,
                  precision=PCP_FP32, lowp_iters=12, d_rank=None,
                  d_scale=None, d_iters=None, stream=None):
    pA, lda = _cm(A, "A")
    check(load().pcp_l1_filter(
        _ptr(M), _ptr(d_pidx), d_pidx.numel(), sp, _ptr(d_qidx),
        d_qidx.numel(), sq, pA, lda, r, _ptr(d_rank), _ptr(d_scale), _ptr(Z),
        ldz, eps, rho, beta0_scale, beta_bar_ratio, max_iter, precision,
        lowp_iters, _ptr(d_iters), _stream(stream)), "pcp_l1_filter")


def pcp_l1_filter_kernel(p, r, precision=PCP_FP32):
    """PCP_KERNEL_SIMT (1) or PCP_KERNEL_TENSOR (2): the Algorithm 1 kernel
    the library runs for problems of length p and rank r."""
    k = load().pcp_l1_filter_kernel(int(p), int(r), int(precision))
    if k < 0:
        check(k, "pcp_l1_filter_kernel")
    return k


def pcp_assemble_factors(U, Sigma, V, d_rank, r, d_rows, d_cols, Lu, Lv, U32,
                         V32, inv_sigma32, stream=None):
    mp, ku = U.shape
    np_ = V.shape[0]
    pLu, ldu = _cm(Lu, "Lu")
    pLv, ldv = _cm(Lv, "Lv")
    check(load().pcp_assemble_factors(
        _ptr(U), _ptr(Sigma), _ptr(V), mp, np_, ku, _ptr(d_rank), r,
        _ptr(d_rows), _ptr(d_cols), pLu, ldu, pLv, ldv, _ptr(U32), _ptr(V32),
        _ptr(inv_sigma32), _stream(stream)), "pcp_assemble_factors")


def pcp_spass(M, Lu, Lv, S, stream=None, impl=None):
    """S = M - Lu Lv^T; impl None (library choice) or PCP_SPASS_AUTO /
    PCP_SPASS_SIMT / PCP_SPASS_TENSOR."""
    pM, ldm = _cm(M, "M")
    pLu, ldu = _cm(Lu, "Lu")
    pLv, ldv = _cm(Lv, "Lv")
    pS, lds = _cm(S, "S")
    m, n = M.shape
    r = Lu.shape[1]
    if impl is None:
        check(load().pcp_spass(pM, ldm, pLu, ldu, pLv, ldv, r, pS, lds, m, n,
                               _stream(stream)), "pcp_spass")
    else:
        check(load().pcp_spass_impl(pM, ldm, pLu, ldu, pLv, ldv, r, pS, lds,
                                    m, n, int(impl), _stream(stream)),
              "pcp_spass_impl")


def solve(M, r, seed_rows=None, seed_cols=None, want_S=True, stream=None,
          raise_on_error=True, **overrides):
    """One-call Algorithm 2: returns (Lu, Lv, S, info, rows, cols).

    ``M`` is a column-major float32 CUDA tensor (m x n).  Keyword overrides
    set pcp_params fields (e.g. filter_tol=1e-6).
    """
    m, n = M.shape
    p = pcp_params_default(m, n, r)
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    plan = Plan(p, seed_rows, seed_cols)
    Lu = colmajor(m, r, device=M.device)
    Lv = colmajor(n, r, device=M.device)
    S = colmajor(m, n, device=M.device) if want_S else None
    st, info, rows, cols = pcp_l1filter_solve(plan, M, Lu, Lv, S, True,
                                              stream, raise_on_error)
    plan.close()
    return Lu, Lv, S, info, rows, cols, st
