"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/mgwr.h declares, and rejects invalid arguments on the host
(no CUDA work is issued by any call made here)."""
import ctypes as C
import math
import os
import re
import shutil

import pytest

from paper_1608_05400_gb300 import mgwr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgwr.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mgwr_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(mgwr.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        from paper_1608_05400_gb300 import _build
        _build.build()
    return mgwr.load()


def test_library_exports_every_declared_function(lib):
    declared = header_functions()
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared set
    assert sorted(mgwr.exported_symbols()) == declared


@pytest.mark.parametrize("args", [
    (3, 63, 64, 1.0, 0.5),      # d
    (1, 62, 64, 1.0, 0.5),      # n not 2^k - 1
    (1, 0, 64, 1.0, 0.5),
    (2, 8191, 64, 1.0, 0.5),    # n too large in 2-D
    (1, 63, 48, 1.0, 0.5),      # M not a power of two
    (1, 63, 2, 1.0, 0.5),       # M too small
    (1, 63, 1 << 21, 1.0, 0.5),  # M too large
    (1, 63, 64, 0.0, 0.5),      # T
    (1, 63, 64, float("inf"), 0.5),
    (1, 63, 64, 1.0, 0.0),      # alpha
    (1, 63, 64, 1.0, 1.5),
    (1, 63, 64, 1.0, float("nan")),
])
def test_create_rejects_invalid_arguments_on_host(lib, args):
    h = C.c_void_p()
    assert lib.mgwr_create(*args, C.byref(h)) == mgwr.MGWR_E_INVAL
    assert not h.value


def test_null_handle_calls_are_rejected(lib):
    assert lib.mgwr_solve(None, 1, 1, 1, 1e-10, 10, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_set_precision(None, 0) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_destroy(None) == mgwr.MGWR_OK
    assert lib.mgwr_last_error(None) == b"null handle"
    assert lib.mgwr_create(1, 63, 64, 1.0, 0.5, None) == mgwr.MGWR_E_INVAL


def test_status_strings(lib):
    for code in range(-9, 1):
        assert lib.mgwr_status_string(code) not in (None, b"unknown status")


def test_footprint_is_host_arithmetic_and_scales(lib):
    from paper_1608_05400_gb300.mgwr import MGWR_FP64, MGWR_MIXED, footprint
    # finest FP64 fields alone: u, f, r, dl of 255^2 x 1024 doubles
    fields = 4 * 255 ** 2 * 1024 * 8
    fp = footprint(2, 255, 1024, 1, MGWR_FP64)
    assert fields < fp < 1.5 * fields
    # mixed keeps the FP64 iterate, right-hand side and carried outer defect and
    # an FP32 hierarchy: about 8 / 7 of FP64 on a 2-D grid
    mx = footprint(2, 255, 1024, 1, MGWR_MIXED)
    assert 3 * 255 ** 2 * 1024 * 8 + 4 * 255 ** 2 * 1024 * 4 < mx < 1.15 * fp
    # linear in the batch, monotone in n and M
    assert abs(footprint(2, 63, 256, 64) - 64 * footprint(2, 63, 256, 1)) < 64 * (3 << 20)
    assert footprint(1, 63, 64) < footprint(1, 127, 64) < footprint(1, 127, 128)
    # long lines (M > 4096) add the partitioned-convolution scratch: 16 bytes per
    # line pair and transform value of the finest level, ceil(N/2) * 2M of them
    n, M = 4095, 65536
    fields = 4 * n * M * 8
    scratch = 16 * ((n + 1) // 2) * 2 * M
    lg = footprint(1, n, M, 1, MGWR_FP64)
    assert 2 * fields + scratch < lg < 2 * fields + scratch + (64 << 20)
    assert footprint(1, 63, 4096) < footprint(1, 63, 8192) < footprint(1, 63, 1 << 20)
    v = C.c_size_t()
    assert lib.mgwr_footprint(2, 64, 256, 1, 0, C.byref(v)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_footprint(2, 63, 256, 0, 0, C.byref(v)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_footprint(2, 63, 256, 1, 7, C.byref(v)) == mgwr.MGWR_E_INVAL


def test_server_calls_reject_null_and_bad_arguments(lib):
    t = C.c_uint64()
    rq = mgwr.mgwr_request()
    assert lib.mgwr_submit(None, C.byref(rq), C.byref(t)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_poll(None, 1, 0, None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_server_destroy(None) == mgwr.MGWR_OK
    h = C.c_void_p()
    assert lib.mgwr_server_create(0, 4, C.byref(h)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_server_set_policy(None, mgwr.MGWR_POLICY_SMALLEST) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_server_create(1 << 30, 0, C.byref(h)) == mgwr.MGWR_E_INVAL
    p = mgwr._dp()
    assert lib.mgwr_server_buffer(None, 16, C.byref(p)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_submit_buffer(None, C.byref(rq), p, C.byref(t)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_server_release(None, p) == mgwr.MGWR_E_INVAL


def test_auto_precision_follows_the_fp32_refinement_limit(lib):
    # 4 eps32 / (pi h)^2 >= 0.2 only from h = 1/4096 on: double-float inner cycles
    # there, the FP32 refinement on coarser grids; host arithmetic only
    from paper_1608_05400_gb300.mgwr import (MGWR_AUTO, MGWR_DD, MGWR_FP64, MGWR_MIXED,
                                             MGWR_MIXED_DD, auto_precision, footprint)
    limit = lambda n: 4 * 2.0 ** -24 / (math.pi / (n + 1)) ** 2
    for d, n in [(1, 63), (1, 1023), (1, 2047), (2, 255), (2, 511), (1, 4095), (1, 8191), (2, 4095)]:
        want = MGWR_DD if limit(n) >= 0.2 else MGWR_MIXED_DD
        assert auto_precision(d, n, 256) == want, (d, n)
        assert footprint(d, n, 256, 1, MGWR_AUTO) == footprint(d, n, 256, 1, want)
    assert auto_precision(1, 2047, 64) == MGWR_MIXED_DD and auto_precision(1, 4095, 64) == MGWR_DD
    for p in (MGWR_FP64, MGWR_MIXED, MGWR_MIXED_DD, MGWR_DD):
        assert auto_precision(1, 4095, 64, p) == p
    r = C.c_int()
    assert lib.mgwr_auto_precision(1, 64, 64, MGWR_AUTO, C.byref(r)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_auto_precision(1, 63, 64, 5, C.byref(r)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_auto_precision(3, 63, 64, MGWR_AUTO, C.byref(r)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_get_precision(None, C.byref(r)) == mgwr.MGWR_E_INVAL


@pytest.mark.parametrize("args", [
    (62, 32, 1.0, 0.5, 1.0, 0),            # n not 2^k - 1
    (0, 32, 1.0, 0.5, 1.0, 0),
    (8191, 32, 1.0, 0.5, 1.0, 0),          # n too large
    (31, 0, 1.0, 0.5, 1.0, 0),             # M too small
    (31, 1025, 1.0, 0.5, 1.0, 0),          # M too large for the direct history sums
    (31, 4097, 1.0, 0.5, 1.0, 0),
    (31, 32, 0.0, 0.5, 1.0, 0),            # T
    (31, 32, math.inf, 0.5, 1.0, 0),
    (31, 32, 1.0, 0.0, 1.0, 0),            # alpha
    (31, 32, 1.0, 1.5, 1.0, 0),
    (31, 32, 1.0, 0.5, math.nan, 0),       # c
    (31, 32, 1.0, 0.5, 1e31, 0),
    (31, 32, 1e-200, 1.0, 1.0, 0),         # L1 scale (T/M)^-alpha / Gamma(2-alpha) > 1e30
    (31, 32, 1.0, 0.5, 1.0, 2),            # coefficient
])
def test_fas_create_rejects_bad_arguments(lib, args):
    h = C.c_void_p()
    assert lib.mgwr_fas_create(*args, C.byref(h)) == mgwr.MGWR_E_INVAL
    assert h.value is None


def test_fas_calls_reject_a_null_handle(lib):
    d = C.c_double()
    i = C.c_int()
    assert lib.mgwr_fas_destroy(None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_set_order(None, 0) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_reset(None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_set_stream(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_set_rhs(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_set_initial(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_solve(None, 1, 0, 1, 1e-10, 10, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_cycle(None, 1, 0, 1) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_residual(None, C.byref(d), None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_get_solution(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_levels(None, C.byref(i)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_smooth(None, 0, 0) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_defect(None, 0, C.byref(d)) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_field_set(None, 0, 0, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_field_get(None, 0, 0, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_fas_last_error(None) == b"null handle"


def test_group_and_set_problem_reject_invalid_arguments_on_host(lib):
    h = C.c_void_p()
    assert lib.mgwr_group_add(None, None, 1, 1, 1, 1e-10, 10) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_group_step(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_group_collect(None, C.byref(h), None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_group_info(None, None, None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_group_destroy(None) == mgwr.MGWR_OK
    assert lib.mgwr_group_create(None) == mgwr.MGWR_E_INVAL
    st = (C.c_int * 1)()
    assert lib.mgwr_group_solve(None, 1, 1, 1, 1, 1e-10, 10, st, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_set_problem(None, None, None) == mgwr.MGWR_E_INVAL


def test_peak_probe_rejects_null_outputs_on_host(lib):
    v = C.c_double()
    assert lib.mgwr_peak_probe(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_peak_probe(C.byref(v), None) == mgwr.MGWR_E_INVAL


def test_device_loop_switch_rejects_a_null_handle(lib):
    assert lib.mgwr_set_device_loop(None, 1) == mgwr.MGWR_E_INVAL


def test_pipelined_transfer_calls_reject_a_null_handle(lib):
    assert lib.mgwr_stage_rhs(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_take_rhs(None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_stage_solution(None, None) == mgwr.MGWR_E_INVAL
    assert lib.mgwr_wait_staged(None) == mgwr.MGWR_E_INVAL
