"""The C-ABI library builds, loads and exports every symbol include/isofft.h
declares; argument validation answers without a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1106_0557_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ipf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ipf_plan_create", "ipf_plan_destroy", "ipf_solve", "ipf_submit_batch",
                     "ipf_greens_cache_bytes", "ipf_greens_cache_trim", "ipf_status_string",
                     "ipf_plan_workspace_bytes", "ipf_solve_host", "ipf_solve_host_async", "ipf_plan_host_wait"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(native.library_path() if os.path.exists(native.library_path()) else native.lib()._name)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # and the binding exposes each under the same name
    for n in declared_functions():
        assert hasattr(native, n), n


def test_status_strings():
    assert native.ipf_status_string(0) == "ok"
    assert native.ipf_status_string(native.IPF_UNSUPPORTED_SIZE) == "unsupported size"
    assert native.ipf_status_string(12345) == "unknown status"


@pytest.mark.parametrize("n,h,dtype,status", [
    ((0, 4, 4), (1.0, 1.0, 1.0), "f32", native.IPF_INVALID_ARG),
    ((4, 4, 4), (1.0, -1.0, 1.0), "f32", native.IPF_INVALID_ARG),
    ((4, 4, 4), (1.0, float("nan"), 1.0), "f64", native.IPF_INVALID_ARG),
    ((4, 4, 4), (1.0, 0.0, 1.0), "f64", native.IPF_INVALID_ARG),
    ((4, 4, 1200), (1.0, 1.0, 1.0), "f32", native.IPF_UNSUPPORTED_SIZE),
    ((2000, 4, 4), (1.0, 1.0, 1.0), "f64", native.IPF_UNSUPPORTED_SIZE),
])
def test_validation_without_gpu(n, h, dtype, status):
    with pytest.raises(native.IsofftError) as ei:
        native.ipf_plan_create(n, h, dtype)
    assert ei.value.status == status
    with pytest.raises(native.IsofftError) as ei:
        native.ipf_estimate_bytes(n, h, dtype)
    assert ei.value.status == status


def test_bad_dtype_and_flags():
    rc = native.lib().ipf_plan_create(ctypes.byref(ctypes.c_void_p()), (ctypes.c_int64 * 3)(4, 4, 4),
                                      (ctypes.c_double * 3)(1, 1, 1), 7, 0, 0, None)
    assert rc == native.IPF_INVALID_ARG
    rc = native.lib().ipf_plan_create(ctypes.byref(ctypes.c_void_p()), (ctypes.c_int64 * 3)(4, 4, 4),
                                      (ctypes.c_double * 3)(1, 1, 1), 0, 1 << 9, 0, None)
    assert rc == native.IPF_INVALID_ARG
    # at most one y-pass form can be forced
    for two in (native.IPF_FLAG_Y_TILES | native.IPF_FLAG_Y_STREAM,
                native.IPF_FLAG_Y_TILES | native.IPF_FLAG_Y_TILES_NARROW,
                native.IPF_FLAG_Y_STREAM | native.IPF_FLAG_Y_TILES_NARROW):
        rc = native.lib().ipf_plan_create(ctypes.byref(ctypes.c_void_p()), (ctypes.c_int64 * 3)(4, 4, 4),
                                          (ctypes.c_double * 3)(1, 1, 1), 0, two, 0, None)
        assert rc == native.IPF_INVALID_ARG
    assert native.lib().ipf_plan_create(None, None, None, 0, 0, 0, None) == native.IPF_INVALID_ARG


def test_null_handles():
    assert native.lib().ipf_plan_destroy(None) == native.IPF_OK
    assert native.lib().ipf_solve(None, None, None, None) == native.IPF_INVALID_ARG
    assert native.lib().ipf_submit_batch(None, 0, None, None, None) == native.IPF_OK
    assert native.lib().ipf_submit_batch(None, 1, None, None, None) == native.IPF_INVALID_ARG
    assert native.lib().ipf_plan_pass_times(None, None) == native.IPF_INVALID_ARG
    assert native.lib().ipf_plan_check(None, None) == native.IPF_INVALID_ARG
    assert native.lib().ipf_plan_variants(None, None) == native.IPF_INVALID_ARG
    assert native.lib().ipf_solve_host_async(None, None, None, None) == native.IPF_INVALID_ARG
    assert native.lib().ipf_plan_host_wait(None) == native.IPF_INVALID_ARG
    assert native.ipf_greens_cache_bytes() >= 0
    assert native.ipf_launch_count() >= 0
