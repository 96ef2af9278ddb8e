"""The C ABI library loads and exports every entry point include/*.h declares.

CPU only: no compute call is made (there is no GPU here); only pure host
entry points (parameter defaults, version, workspace sizing, argument
validation before any device work) are exercised.
"""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1108_5359_gb300 import build, _abi
    build.build()
    return _abi.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pcp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pcp_l1filter_solve" in names and "pcp_spass" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_python_prototypes_cover_header():
    from paper_1108_5359_gb300 import _abi
    assert _declared() == set(_abi.PROTOTYPES)


def test_params_default_values(lib):
    from paper_1108_5359_gb300 import pcp_params_default
    p = pcp_params_default(5000, 5000, 20)
    assert (p.m, p.n, p.r) == (5000, 5000, 20)
    assert p.s_r == 10.0 and p.s_c == 10.0      # Section 3.1
    assert p.seed_tol == 1e-7                   # Section 4.1.1
    assert p.filter_rho > 1 and p.filter_tol > 0  # Algorithm 1 constraints
    assert lib.pcp_params_default(None, 1, 1, 1) == -1


def test_version_and_workspace(lib):
    assert b"sm_103a" in lib.pcp_version()
    assert lib.pcp_seed_workspace_bytes(200, 200, 52) > 4 * 200 * 200 * 8
    assert lib.pcp_seed_workspace_bytes(0, 200, 52) == 0


def test_plan_rejects_bad_arguments_without_gpu(lib):
    # validation happens before any device call
    from paper_1108_5359_gb300 import _abi, pcp_params_default
    p = pcp_params_default(100, 100, 0)
    h = C.c_void_p()
    assert lib.pcp_l1filter_plan(C.byref(p), C.byref(h)) == _abi.PCP_ERR_ARG
    assert b"r=0" in lib.pcp_last_error()
    p = pcp_params_default(100, 100, 20)   # seed 200 x 200 > 100 x 100
    assert lib.pcp_l1filter_plan(C.byref(p), C.byref(h)) == _abi.PCP_ERR_ARG
    p = pcp_params_default(1000, 1000, 5)
    bad = (C.c_int64 * 50)(*([3] * 50))     # repeated index
    p.seed_rows = C.cast(bad, C.POINTER(C.c_int64))
    assert lib.pcp_l1filter_plan(C.byref(p), C.byref(h)) == _abi.PCP_ERR_ARG
    assert b"repeated" in lib.pcp_last_error()


def test_stage_entry_points_validate_sizes(lib):
    from paper_1108_5359_gb300 import _abi
    # p out of range -> PCP_ERR_ARG before any launch
    st = lib.pcp_l1_filter(None, None, 0, 1, None, 4, 1, None, 1, 4, None,
                           None, None, 1, 1e-6, 1.5, 1.0, 1e10, 10, 0, 0,
                           None, None)
    assert st == _abi.PCP_ERR_ARG
    st = lib.pcp_spass(None, 1, None, 1, None, 1, 100, None, 1, 1, 1, None)
    assert st == _abi.PCP_ERR_ARG


def test_seed_entry_point_limits(lib):
    # the seed stage's size limits are refused before any device work: sides
    # in [2, 512], kmax even, <= 64 and <= the short side, k0 even in
    # [2, kmax]; a valid shape with null buffers is refused too
    from paper_1108_5359_gb300 import _abi

    def call(mp, np_, k0, kmax):
        return lib.pcp_seed_pcp(None, mp, np_, 0.0, 1e-7, 1.5, 1.25, 1e7,
                                10, k0, kmax, 1e-6, 0, None, None, None,
                                None, None, None, None, None)

    for mp, np_, k0, kmax, what in [(513, 100, 8, 8, "outside"),
                                    (100, 513, 8, 8, "outside"),
                                    (1, 100, 2, 2, "outside"),
                                    (512, 512, 8, 66, "kmax"),
                                    (512, 512, 8, 7, "kmax"),
                                    (512, 7, 8, 8, "kmax"),
                                    (512, 8, 8, 10, "kmax"),
                                    (512, 512, 10, 8, "k0"),
                                    (512, 512, 3, 8, "k0"),
                                    (512, 512, 60, 64, "null"),
                                    (512, 8, 8, 8, "null"),
                                    (512, 7, 6, 6, "null")]:
        assert call(mp, np_, k0, kmax) == _abi.PCP_ERR_ARG, (mp, np_, kmax)
        assert what in lib.pcp_last_error().decode()
    assert lib.pcp_seed_workspace_bytes(512, 512, 64) > 0
    assert lib.pcp_seed_workspace_bytes(0, 512, 64) == 0


def test_batch_and_serve_validate_without_gpu(lib):
    from paper_1108_5359_gb300 import _abi
    assert lib.pcp_l1filter_batch(0, None, None, None) == _abi.PCP_OK
    assert lib.pcp_l1filter_batch(-1, None, None, None) == _abi.PCP_ERR_ARG
    assert lib.pcp_l1filter_batch(2, None, None, None) == _abi.PCP_ERR_ARG
    h = C.c_void_p()
    assert lib.pcp_serve_create(0, 4, 1, C.byref(h)) == _abi.PCP_ERR_ARG
    assert lib.pcp_serve_create(1 << 30, 0, 1, C.byref(h)) == _abi.PCP_ERR_ARG
    assert lib.pcp_serve_create(1 << 30, 4, 17, C.byref(h)) == _abi.PCP_ERR_ARG
    assert not h.value
    assert lib.pcp_serve_destroy(None) == _abi.PCP_OK
    assert lib.pcp_serve_poll(None, 1, None) == _abi.PCP_ERR_ARG
    assert lib.pcp_serve_stop(None) == _abi.PCP_ERR_ARG


def test_new_entry_points_validate_without_gpu(lib):
    from paper_1108_5359_gb300 import _abi
    # S-pass kernel choice: unknown choice and out-of-range rank refused
    # before any device work; an empty matrix is a no-op
    st = lib.pcp_spass_impl(None, 1, None, 1, None, 1, 4, None, 1, 1, 1, 7,
                            None)
    assert st == _abi.PCP_ERR_ARG
    st = lib.pcp_spass_impl(None, 1, None, 1, None, 1, 65, None, 1, 1, 1, 0,
                            None)
    assert st == _abi.PCP_ERR_ARG
    st = lib.pcp_spass_impl(None, 1, None, 1, None, 1, 4, None, 1, 0, 5, 2,
                            None)
    assert st == _abi.PCP_OK
    # host-buffer solve: null plan / buffers refused
    st = lib.pcp_l1filter_solve_host(None, None, 1, None, None, None, 1,
                                     None, None)
    assert st == _abi.PCP_ERR_ARG
    assert lib.pcp_plan_graph_launches(None) == 0


def test_precision_forms_of_algorithm_1(lib):
    from paper_1108_5359_gb300 import _abi
    # every built precision passes validation (N = 0: no launch); the
    # reserved FP64 form reports PCP_ERR_UNSUPPORTED
    for prec, want in [(0, _abi.PCP_OK), (1, _abi.PCP_OK), (2, _abi.PCP_OK),
                       (3, _abi.PCP_ERR_UNSUPPORTED), (4, _abi.PCP_OK),
                       (5, _abi.PCP_OK), (6, _abi.PCP_ERR_ARG)]:
        st = lib.pcp_l1_filter(None, None, 16, 1, None, 0, 1, None, 16, 4,
                               None, None, None, 1, 1e-6, 1.5, 1.0, 1e10, 10,
                               prec, 4, None, None)
        assert st == want, (prec, st)


def test_filter_kernel_choice_is_a_function_of_the_shape(lib):
    # the PCP_FP32 kernel comes from the compiled-in tuning table: a host
    # lookup, the same answer on every call and in every process
    from paper_1108_5359_gb300 import _abi
    k = lib.pcp_l1_filter_kernel
    for p, r in ((50, 5), (200, 20), (250, 25), (256, 32)):
        got = {k(p, r, _abi.PCP_FP32) for _ in range(3)}
        assert len(got) == 1
        assert got.pop() in (_abi.PCP_KERNEL_SIMT, _abi.PCP_KERNEL_TENSOR)
    # shapes only one kernel takes, and the explicit forms
    assert k(500, 50, _abi.PCP_FP32) == _abi.PCP_KERNEL_TENSOR
    assert k(200, 40, _abi.PCP_FP32) == _abi.PCP_KERNEL_TENSOR
    assert k(200, 20, _abi.PCP_FP32_SIMT) == _abi.PCP_KERNEL_SIMT
    assert k(200, 20, _abi.PCP_FP32_TENSOR) == _abi.PCP_KERNEL_TENSOR
    assert k(200, 20, _abi.PCP_BF16_REFINED) == _abi.PCP_KERNEL_TENSOR
    assert k(600, 20, _abi.PCP_FP32) == _abi.PCP_ERR_ARG
    assert k(300, 20, _abi.PCP_FP32_SIMT) == _abi.PCP_ERR_ARG
    assert k(200, 20, _abi.PCP_FP64) == _abi.PCP_ERR_ARG


def test_table_written_by_the_tuning_run_is_well_formed():
    text = open(os.path.join(ROOT, "paper_1108_5359_gb300", "csrc",
                             "filter_table.inc")).read()
    rows = re.findall(r"\{\s*([12])\s*,\s*([12])\s*,\s*([12])\s*,\s*([12])\s*\}",
                      text)
    assert len(rows) == 3


def test_binding_sizes_the_seed_from_its_index_arrays(lib):
    # a seed index set sets seed_m / seed_n to its length (the library reads
    # that many entries); a size already set to another value is refused;
    # the order arrays of seed growth do not size the seed
    import numpy as np
    import paper_1108_5359_gb300 as pk
    p = pk.pcp_params_default(1000, 900, 5)
    assert p.seed_m == 0 and p.seed_n == 0
    keep = []
    pk._set_index_arrays(p, keep, np.arange(64), np.arange(0, 120, 2),
                         None, None)
    assert (p.seed_m, p.seed_n) == (64, 60)
    assert p.seed_rows[63] == 63 and p.seed_cols[59] == 118
    q = pk.pcp_params_default(1000, 900, 5)
    q.seed_m = 50
    with pytest.raises(ValueError):
        pk._set_index_arrays(q, [], np.arange(64), None, None, None)
    g = pk.pcp_params_default(1000, 900, 5)
    pk._set_index_arrays(g, [], None, None, np.arange(1000), np.arange(900))
    assert (g.seed_m, g.seed_n) == (0, 0)
