"""ctypes declarations of the C ABI in include/pcp_l1f.h.

Argument marshalling only: every computation happens in the CUDA library.
Loading fails loudly when the shared library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

PCP_OK = 0
PCP_ERR_ARG = -1
PCP_ERR_NOMEM = -2
PCP_ERR_CUDA = -3
PCP_ERR_NONFINITE = -4
PCP_ERR_RANK_TEST = -5
PCP_ERR_SEED_NOCONV = -6
PCP_ERR_FILTER_NOCONV = -7
PCP_ERR_BUSY = -8
PCP_ERR_TIMEOUT = -9
PCP_ERR_CANCELLED = -10
PCP_ERR_UNSUPPORTED = -11

STATUS_NAMES = {
    0: "PCP_OK", -1: "PCP_ERR_ARG", -2: "PCP_ERR_NOMEM", -3: "PCP_ERR_CUDA",
    -4: "PCP_ERR_NONFINITE", -5: "PCP_ERR_RANK_TEST",
    -6: "PCP_ERR_SEED_NOCONV", -7: "PCP_ERR_FILTER_NOCONV",
    -8: "PCP_ERR_BUSY", -9: "PCP_ERR_TIMEOUT", -10: "PCP_ERR_CANCELLED",
    -11: "PCP_ERR_UNSUPPORTED",
}

PCP_FP32 = 0
PCP_BF16_REFINED = 1
PCP_TF32_REFINED = 2
PCP_FP64 = 3
PCP_FP32_TENSOR = 4
PCP_FP32_SIMT = 5

PCP_KERNEL_SIMT = 1
PCP_KERNEL_TENSOR = 2
KERNEL_NAMES = {PCP_KERNEL_SIMT: "adm_f32_kernel",
                PCP_KERNEL_TENSOR: "adm_tc_kernel"}

PCP_SPASS_AUTO = 0
PCP_SPASS_SIMT = 1
PCP_SPASS_TENSOR = 2


class PCPParams(C.Structure):
    _fields_ = [
        ("m", C.c_int64), ("n", C.c_int64),
        ("r", C.c_int32), ("precision", C.c_int32),
        ("lambda_", C.c_double), ("lambda_seed", C.c_double),
        ("s_r", C.c_double), ("s_c", C.c_double),
        ("seed_tol", C.c_double), ("seed_rho", C.c_double),
        ("seed_mu_scale", C.c_double), ("seed_mu_max_ratio", C.c_double),
        ("rank_cut", C.c_double),
        ("filter_tol", C.c_double), ("filter_rho", C.c_double),
        ("beta0_scale", C.c_double), ("beta_bar_ratio", C.c_double),
        ("seed_max_iter", C.c_int32), ("filter_max_iter", C.c_int32),
        ("seed_subspace", C.c_int32), ("lowp_iters", C.c_int32),
        ("rng_seed", C.c_uint64),
        ("seed_rows", C.POINTER(C.c_int64)),
        ("seed_cols", C.POINTER(C.c_int64)),
        ("row_order", C.POINTER(C.c_int64)),
        ("col_order", C.POINTER(C.c_int64)),
        ("seed_m", C.c_int32), ("seed_n", C.c_int32),
        ("grow_seed", C.c_int32), ("seed_ctas", C.c_int32),
        ("wait_timeout_ns", C.c_int64),
    ]


class PCPInfo(C.Structure):
    _fields_ = [
        ("rank", C.c_int32), ("rank_ok", C.c_int32),
        ("seed_iters", C.c_int32), ("filter_iters_max", C.c_int32),
        ("seed_m", C.c_int64), ("seed_n", C.c_int64),
        ("problems", C.c_int64), ("problems_unconverged", C.c_int64),
        ("seed_residual", C.c_double), ("lambda_", C.c_double),
        ("t_seed_ms", C.c_float), ("t_filter_ms", C.c_float),
        ("t_spass_ms", C.c_float), ("t_total_ms", C.c_float),
        ("status", C.c_int32), ("seed_rank_raw", C.c_int32),
        ("filter_iters_mean", C.c_double),
        ("filter_kernel", C.c_int32), ("launches", C.c_int32),
        ("seed_team", C.c_int32), ("pad_info", C.c_int32),
    ]

    def as_dict(self):
        return {f[0].rstrip("_"): getattr(self, f[0]) for f in self._fields_}


class PCPProblem(C.Structure):
    _fields_ = [
        ("params", PCPParams),
        ("dM", C.c_void_p), ("ldm", C.c_int64),
        ("dLu", C.c_void_p), ("dLv", C.c_void_p),
        ("dS", C.c_void_p), ("lds", C.c_int64),
    ]


_vp = C.c_void_p
_i32, _i64, _f64 = C.c_int32, C.c_int64, C.c_double
_ip32 = C.POINTER(C.c_int32)
_ip64 = C.POINTER(C.c_int64)
_dp = C.POINTER(C.c_double)

# name -> (restype, argtypes); mirrors include/pcp_l1f.h
PROTOTYPES = {
    "pcp_params_default": (_i32, [C.POINTER(PCPParams), _i64, _i64, _i32]),
    "pcp_last_error": (C.c_char_p, []),
    "pcp_version": (C.c_char_p, []),
    "pcp_l1filter_plan": (_i32, [C.POINTER(PCPParams), C.POINTER(_vp)]),
    "pcp_l1filter_solve": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _ip64,
                                  _ip64, C.POINTER(PCPInfo), _vp]),
    "pcp_plan_destroy": (None, [_vp]),
    "pcp_l1filter_batch": (_i32, [_i32, C.POINTER(PCPProblem),
                                  C.POINTER(PCPInfo), _vp]),
    "pcp_l1filter_batch_plan": (_i32, [_i32, C.POINTER(PCPProblem), _vp,
                                       C.POINTER(_vp)]),
    "pcp_l1filter_batch_run": (_i32, [_vp, C.POINTER(PCPInfo), _vp]),
    "pcp_batch_plan_destroy": (None, [_vp]),
    "pcp_serve_create": (_i32, [C.c_size_t, _i32, _i32, C.POINTER(_vp)]),
    "pcp_serve_submit": (_i32, [_vp, C.POINTER(PCPProblem),
                                C.POINTER(C.c_uint64)]),
    "pcp_serve_poll": (_i32, [_vp, C.c_uint64, C.POINTER(PCPInfo)]),
    "pcp_serve_wait": (_i32, [_vp, C.c_uint64, C.POINTER(PCPInfo)]),
    "pcp_serve_stop": (_i32, [_vp]),
    "pcp_serve_destroy": (_i32, [_vp]),
    "pcp_gather_seed": (_i32, [_vp, _i64, _vp, _i32, _vp, _i32, _vp, _vp]),
    "pcp_seed_workspace_bytes": (C.c_size_t, [_i32, _i32, _i32]),
    "pcp_seed_pcp": (_i32, [_vp, _i32, _i32, _f64, _f64, _f64, _f64, _f64,
                            _i32, _i32, _i32, _f64, _i32, _vp, _vp, _vp, _vp,
                            _ip32, _ip32, _dp, _vp]),
    "pcp_seed_pcp_static": (_i32, [_vp, _i32, _i32, _f64, _f64, _f64, _f64,
                                   _f64, _i32, _i32, _i32, _f64, _i32, _vp,
                                   _vp, _vp, _ip32, _ip32, _dp, _vp]),
    "pcp_seed_trace": (_i32, [_vp, _i32, _i32, _i32, C.POINTER(C.c_uint64),
                              _i32, _vp]),
    "pcp_plan_seed_trace": (_i32, [_vp, C.POINTER(C.c_uint64), _i32, _vp]),
    "pcp_l1_filter": (_i32, [_vp, _vp, _i32, _i64, _vp, _i32, _i64, _vp, _i32,
                             _i32, _vp, _vp, _vp, _i64, _f64, _f64, _f64, _f64,
                             _i32, _i32, _i32, _vp, _vp]),
    "pcp_l1_filter_kernel": (_i32, [_i32, _i32, _i32]),
    "pcp_assemble_factors": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _i32,
                                    _vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp,
                                    _vp, _vp]),
    "pcp_spass": (_i32, [_vp, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _i64,
                         _i64, _i64, _vp]),
    "pcp_plan_graph_launches": (_i64, [_vp]),
    "pcp_l1filter_solve_host": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _i64,
                                       _vp, _vp]),
    "pcp_spass_impl": (_i32, [_vp, _i64, _vp, _i64, _vp, _i64, _i32, _vp,
                              _i64, _i64, _i64, _i32, _vp]),
}

_lib = None


class PCPError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


def lib_path() -> str:
    return LIB


def load():
    """Load libpcpl1f.so (built by paper_1108_5359_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(
            f"{LIB} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    msg = load().pcp_last_error()
    return msg.decode() if msg else ""


def check(status: int, what: str = "") -> int:
    if status != PCP_OK:
        raise PCPError(status, f"{what}: {last_error()}")
    return status
