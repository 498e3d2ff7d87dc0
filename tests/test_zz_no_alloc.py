"""sgl_forward_noalloc: the forward transform for callers that cannot
allocate device memory (scratch and tables in static device arrays of the
library).  It must give what sgl_forward gives on a plan of the same B and
batch, call after call, and refuse requests larger than its static scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1604_05140_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12  # the FP64 tolerance of the parity tests


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
