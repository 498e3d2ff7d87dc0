"""Host-side checks of the C ABI: the library builds, loads, exports every
function include/sgl.h declares, and rejects bad arguments before touching the
GPU (no compute calls: this file runs without a GPU)."""
import ctypes
import os
import subprocess

import pytest

from paper_1604_05140_gb300 import sgl


@pytest.fixture(scope="module")
def lib():
    from paper_1604_05140_gb300 import build
    if build.stale():
        build.build()
    return sgl.load_library()


def test_header_declares_the_boundary():
    names = sgl.header_functions()
    for must in ["sgl_plan", "sgl_plan_many", "sgl_forward", "sgl_inverse", "sgl_adjoint",
                 "sgl_grid", "sgl_destroy", "sgl_last_error", "sgl_check"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", sgl.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in sgl.header_functions() if n not in exported]
    assert not missing, missing
    for n in sgl.header_functions():
        assert hasattr(lib, n)


def test_version(lib):
    assert lib.sgl_version().decode().startswith("sgl-gb300")


@pytest.mark.parametrize("args,status", [
    ((0, 1, 0, 0), sgl.SGL_ERR_ARG),        # B < 1
    ((8, 0, 0, 0), sgl.SGL_ERR_ARG),        # batch < 1
    ((8, 1, 9, 0), sgl.SGL_ERR_ARG),        # unknown precision
    ((6, 1, 2, 0), sgl.SGL_ERR_UNSUPPORTED),    # tensor-core plans need 4 | B
    ((6, 1, 4, 0), sgl.SGL_ERR_UNSUPPORTED),
    ((8, 1, 0, 5), sgl.SGL_ERR_ARG),        # unknown sample convention
    ((8, 1, 1, 1), sgl.SGL_ERR_ARG),        # physical samples need FP64
    ((17, 1, 0, 0), sgl.SGL_ERR_UNSUPPORTED),   # 2B = 2 * 17: odd factor > 16
    ((129, 1, 0, 0), sgl.SGL_ERR_UNSUPPORTED),  # above SGL_MAX_B
])
def test_plan_argument_errors(lib, args, status):
    h = ctypes.c_void_p(1234)
    st = lib.sgl_plan(ctypes.byref(h), *args)
    assert st == status
    assert h.value is None
    assert lib.sgl_last_error(None)


@pytest.mark.parametrize("args,status", [
    ((8, 1, 0, 0, 7), sgl.SGL_ERR_ARG),             # unknown radial grid
    ((6, 1, 2, 0, 1), sgl.SGL_ERR_UNSUPPORTED),     # tensor-core plans: B divisible by 4
    ((6, 3, 3, 2, 1), sgl.SGL_ERR_UNSUPPORTED),     # ... real functions on the paper's grid too
    ((17, 2, 0, 2, 1), sgl.SGL_ERR_UNSUPPORTED),    # unsupported bandlimit, real functions
    ((8, 0, 3, 2, 1), sgl.SGL_ERR_ARG),             # empty batch
    ((8, 1, 1, 1, 1), sgl.SGL_ERR_ARG),             # physical samples still need FP64
    ((0, 1, 0, 0, 1), sgl.SGL_ERR_ARG),
])
def test_plan_grid_argument_errors(lib, args, status):
    h = ctypes.c_void_p(1234)
    assert lib.sgl_plan_grid(ctypes.byref(h), *args) == status
    assert h.value is None
    assert lib.sgl_last_error(None)


def test_creation_errors_are_per_thread(lib):
    # two threads fail plan creation in turn; each then reads its own message
    import threading
    bar = threading.Barrier(2)
    seen = {}

    def worker(name, args):
        h = ctypes.c_void_p()
        if name == "second":
            bar.wait()
        assert lib.sgl_plan(ctypes.byref(h), *args) != sgl.SGL_OK
        if name == "first":
            bar.wait()
        bar.wait()
        seen[name] = lib.sgl_last_error(None).decode()

    t1 = threading.Thread(target=worker, args=("first", (0, 1, 0, 0)))
    t2 = threading.Thread(target=worker, args=("second", (8, 1, 9, 0)))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert "bandlimit" in seen["first"]
    assert "precision" in seen["second"]


def test_midpoint_argument_errors(lib):
    # found before any device call: bandlimit, sizes, precision, null pointers
    assert lib.sgl_midpoint(0, 8, 5.0, 1, 0, None, None, None) == sgl.SGL_ERR_UNSUPPORTED
    assert lib.sgl_midpoint(33, 8, 5.0, 1, 0, None, None, None) == sgl.SGL_ERR_UNSUPPORTED
    assert lib.sgl_midpoint(4, 0, 5.0, 1, 0, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_midpoint(4, 8, 0.0, 1, 0, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_midpoint(4, 8, 5.0, 0, 0, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_midpoint(4, 8, 5.0, 1, 2, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_midpoint(4, 8, 5.0, 1, 0, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_last_error(None)


def test_plan_many_argument_errors(lib):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * 3)(8, 0, 16)
    assert lib.sgl_plan_many(ctypes.byref(h), arr, 3, 2) == sgl.SGL_ERR_ARG
    assert lib.sgl_plan_many(ctypes.byref(h), arr, 0, 2) == sgl.SGL_ERR_ARG
    assert lib.sgl_plan_many(None, arr, 3, 2) == sgl.SGL_ERR_ARG


def test_null_plan_queries(lib):
    assert lib.sgl_set_dlt(None, 1) == sgl.SGL_ERR_ARG
    assert lib.sgl_radii(None, 0) == -1
    assert lib.sgl_sample_count(None) == -1
    assert lib.sgl_coeff_offset(None, 0) == -1
    assert lib.sgl_forward(None, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_autotune(None, None, None, None, None) == sgl.SGL_ERR_ARG
    assert lib.sgl_tuning(None) == b""
    assert lib.sgl_set_graphs(None, 1) == sgl.SGL_ERR_ARG
    lib.sgl_destroy(None)


def test_binding_has_every_function_under_its_own_name(lib):
    # the Python binding exposes each C function of the header as a module
    # function of the same name; plan-free and null-plan calls need no GPU
    missing = [n for n in sgl.header_functions() if not callable(getattr(sgl, n, None))]
    assert not missing, missing
    assert sgl.sgl_version().startswith("sgl-gb300")
    assert [sgl.sgl_stage_name(k) for k in range(sgl.SGL_NUM_STAGES)] == [
        "fft_forward", "legendre_forward", "radial_forward", "radial_inverse", "legendre_inverse", "fft_inverse"]
    assert sgl.sgl_stage_name(sgl.SGL_NUM_STAGES) == ""
    for q in (sgl.sgl_sample_count, sgl.sgl_coeff_count, sgl.sgl_num_functions, sgl.sgl_workspace_bytes,
              sgl.sgl_launches_per_call, sgl.sgl_graph_count):
        assert q(None) == -1
    for q in (sgl.sgl_sample_offset, sgl.sgl_coeff_offset, sgl.sgl_bandlimit, sgl.sgl_radii):
        assert q(None, 0) == -1
    for call in (lambda: sgl.sgl_set_profiling(None, True), lambda: sgl.sgl_stage_times(None),
                 lambda: sgl.sgl_set_dlt(None, True), lambda: sgl.sgl_forward_noalloc(8, 0, 1, 1)):
        with pytest.raises(sgl.SGLError) as e:
            call()
        assert e.value.status == sgl.SGL_ERR_ARG
    with pytest.raises(sgl.SGLError) as e:
        sgl.sgl_forward_noalloc(0, 1, 1, 1)
    assert e.value.status == sgl.SGL_ERR_UNSUPPORTED
    assert "bandlimits" in sgl.sgl_last_error(None)


def test_selftest_wait_argument_errors(lib):
    import ctypes
    flag = ctypes.c_int(7)
    assert lib.sgl_selftest_wait(0, ctypes.byref(flag)) == sgl.SGL_ERR_ARG            # no bound
    assert lib.sgl_selftest_wait(3_000_000_000, ctypes.byref(flag)) == sgl.SGL_ERR_ARG  # above 2 s
    assert lib.sgl_selftest_wait(1000, None) == sgl.SGL_ERR_ARG


def test_supported_bandlimits_match_header_rule():
    # every B <= 16 and every multiple of 8 up to 128 (the header's rule)
    from paper_1604_05140_gb300.inputs import uneven_bandlimits
    for B in list(range(1, 17)) + list(range(8, 129, 8)):
        n = 2 * B
        p = 1
        while p < 16 and n % (2 * p) == 0:
            p *= 2
        assert n // p <= 16, B
    assert set(uneven_bandlimits()) <= set(range(16, 129, 8))
    # the complete set: also these bandlimits that are neither <= 16 nor multiples of 8
    extra = []
    for B in range(17, 129):
        n, p = 2 * B, 1
        while p < 16 and n % (2 * p) == 0:
            p *= 2
        if n // p <= 16 and B % 8:
            extra.append(B)
    assert extra == [18, 20, 22, 26, 28, 30, 36, 44, 52, 60]
