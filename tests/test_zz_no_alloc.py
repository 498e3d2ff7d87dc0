"""sgl_forward_noalloc: the forward transform for callers that cannot
allocate device memory (scratch and tables in static device arrays of the
library).  It must give what sgl_forward gives on a plan of the same B and
batch, call after call; agree with the FP64 oracle with its own launch
schedule, up to the largest batch its scratch holds; leave the device's free
memory unchanged on a repeated call; and refuse requests larger than its
static scratch, host pointers and other devices' pointers.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12  # the FP64 tolerance of the parity tests
SCRATCH_DOUBLES = 2 ** 21  # the static scratch


def _largest_batch(B):
    # E/O spectra 4 B^2 (2B - 1) plus per-degree spectra 2 B^3 doubles per function
    return SCRATCH_DOUBLES // (4 * B * B * (2 * B - 1) + 2 * B ** 3)


def _call(lib, B, batch, g, out):
    vp = ctypes.c_void_p
    return lib.sgl_forward_noalloc(B, batch, vp(g.data_ptr()), vp(out.data_ptr()), vp(_stream()))


def _lib():
    from paper_1604_05140_gb300 import sgl
    return sgl.load_library()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def test_noalloc_forward_matches_plan_forward_on_consecutive_calls():
    from paper_1604_05140_gb300 import Plan
    lib = _lib()
    # (8, 3) twice, then (16, 2) twice (tables re-uploaded), then (8, 3) again
    for B, batch, seeds in [(8, 3, (1, 2)), (16, 2, (3, 4)), (8, 3, (5, 6))]:
        plan = Plan(B, batch, "fp64")
        for seed in seeds:
            g = torch.from_numpy(inputs.random_samples(B, batch, seed=seed)).cuda()
            ref = plan.forward(g)
            out = torch.full(plan.coeff_shape, float("nan"), dtype=torch.complex128, device="cuda")
            st = lib.sgl_forward_noalloc(B, batch, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(_stream()))
            assert st == 0, lib.sgl_last_error(None)
            torch.cuda.synchronize()
            err = ((out - ref).abs().max() / ref.abs().max()).item()
            assert err < FP64_TOL, (B, batch, seed, err)
        plan.close()


def test_noalloc_rejects_what_it_cannot_hold():
    lib = _lib()
    g = torch.zeros(8, dtype=torch.complex128, device="cuda")
    out = torch.zeros(8, dtype=torch.complex128, device="cuda")
    vp = ctypes.c_void_p
    # B = 32 fits 6 functions in the static scratch, not 7
    st = lib.sgl_forward_noalloc(32, 7, vp(g.data_ptr()), vp(out.data_ptr()), vp(_stream()))
    assert st == 5 and b"scratch" in lib.sgl_last_error(None)
    st = lib.sgl_forward_noalloc(64, 1, vp(g.data_ptr()), vp(out.data_ptr()), vp(_stream()))
    assert st == 5
    # host buffers would need staging memory
    host = np.zeros(4 * 8 ** 3, dtype=np.complex128)
    st = lib.sgl_forward_noalloc(8, 1, vp(host.ctypes.data), vp(out.data_ptr()), vp(_stream()))
    assert st == 1


@pytest.mark.parametrize("B", [1, 8, 32])
def test_noalloc_forward_vs_oracle_at_largest_batch(B):
    # this entry point has its own launch schedule (64 x 64 SIMT tiles only):
    # check it against the oracle's forward directly, at the largest batch its
    # scratch accepts (B = 8: 431 functions, B = 32: 6).  At B = 1 the launch
    # schedules reach the 8 MiB table region first (the scratch would hold
    # 349525 functions): that batch is refused, 100000 functions run.
    lib = _lib()
    batch = _largest_batch(B)
    one = torch.zeros(1, dtype=torch.complex128, device="cuda")
    assert _call(lib, B, batch + 1, one, one) == 5
    if B == 1:
        big_g = torch.zeros((batch, 4), dtype=torch.complex128, device="cuda")
        big_out = torch.zeros((batch, 1), dtype=torch.complex128, device="cuda")
        assert _call(lib, B, batch, big_g, big_out) == 5
        assert b"exceed" in lib.sgl_last_error(None)
        del big_g, big_out
        batch = 100000
    g_np = inputs.random_samples(B, batch, seed=31 + B)
    g = torch.from_numpy(g_np).cuda()
    out = torch.full((batch, O.coeff_count(B)), float("nan"), dtype=torch.complex128, device="cuda")
    for _ in range(2):  # twice in a row: the second call reuses the uploaded tables
        assert _call(lib, B, batch, g, out) == 0, lib.sgl_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # every function checked when the oracle is cheap, else a spread sample
        idx = np.arange(batch) if batch <= 512 else np.linspace(0, batch - 1, 512).astype(int)
        ref = O.forward(g_np[idx], B)
        err = (np.abs(got[idx] - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()
        assert err < FP64_TOL, (B, batch, err)
        out.fill_(float("nan"))


def test_noalloc_repeated_call_reserves_no_device_memory():
    # after the first call with a given (B, batch), a second one changes
    # nothing in the device's free memory
    lib = _lib()
    B, batch = 16, 8
    g = torch.from_numpy(inputs.random_samples(B, batch, seed=77)).cuda()
    out = torch.empty((batch, O.coeff_count(B)), dtype=torch.complex128, device="cuda")
    assert _call(lib, B, batch, g, out) == 0, lib.sgl_last_error(None)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _call(lib, B, batch, g, out) == 0, lib.sgl_last_error(None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
