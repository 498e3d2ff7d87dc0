"""Failure detection without a GPU fault.

Every wait of the tensor-core kernels on an mbarrier is bounded; a wait that
gives up sets the plan's error flag and ends its kernel, and sgl_check reports
SGL_ERR_TIMEOUT.  sgl_selftest_wait runs the same bounded wait on a barrier
that nothing completes (a flag that nothing sets), with a 50 ms bound: the
wait must give up, the kernel must end, and the CUDA context must stay usable
for a transform afterwards.
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs
from tolerances import SPLIT_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    from paper_1604_05140_gb300 import Plan, sgl_selftest_wait
    t0 = time.perf_counter()
    assert sgl_selftest_wait(50_000_000) is True
    assert time.perf_counter() - t0 < 5.0           # the bound, not a hang
    # the context still runs the tensor-core path correctly
    B = 16
    p = Plan(B, 2, "tf32x3")
    c = inputs.random_coeffs(B, 2, seed=4242)
    s = p.inverse(torch.from_numpy(c).to(torch.complex64).cuda()).cpu().numpy()
    ref = O.inverse(c, B)
    assert np.abs(s - ref).max() / np.abs(ref).max() < SPLIT_TOL
    p.check()                                          # this plan's flag is clear
