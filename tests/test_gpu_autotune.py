"""Autotuner (sgl_autotune): timing-based choice of the launch configuration,
its cache file, and unchanged results.

A TF32x3 plan of B=64 x 4 functions is tuned with a cache file; the chosen
configuration must be one of the candidates, the transform must still agree
with the FP64 oracle within the TF32x3 bound, and a second plan of the same
shape must pick the configuration up from the cache without timing.
"""
import re

import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tolerances import SPLIT_TOL as TF32X3_TOL


def _parse(text):
    m = re.match(r"fft_fwd_jp=(\d+) fft_inv_jp=(\d+) rad_inv_narrow=(\d+) source=(\w+)", text)
    assert m, text
    return int(m.group(1)), int(m.group(2)), int(m.group(3)), m.group(4)


def test_autotune_cache_and_parity(tmp_path):
    from paper_1604_05140_gb300 import Plan
    B, NB = 64, 4
    cache = str(tmp_path / "tuning.txt")
    plan = Plan(B, NB, "tf32x3")
    assert _parse(plan.tuning)[3] == "default"
    jf, ji, rn, src = _parse(plan.autotune(cache=cache))
    assert src == "timed" and jf in (4, 8, 16) and ji in (4, 8, 16) and rn in (1, 65)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and f"segs={B}x{NB}," in lines[0]

    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 3, decay=True)
    ct = torch.from_numpy(c).to(torch.complex64).cuda()
    s = plan.inverse(ct)
    f = plan.forward(s).cpu().numpy()
    ref = O.inverse(c[:1], B)
    s0 = s[:1].cpu().numpy()
    assert np.abs(s0 - ref).max() / np.abs(ref).max() < TF32X3_TOL
    assert np.abs(f - c).max() / np.abs(c).max() < TF32X3_TOL
    plan.check()

    plan2 = Plan(B, NB, "tf32x3")
    assert _parse(plan2.autotune(cache=cache)) == (jf, ji, rn, "cache")
    assert len(open(cache).read().splitlines()) == 1
    f2 = plan2.forward(plan2.inverse(ct)).cpu().numpy()
    assert np.array_equal(f, f2)  # same configuration, same arithmetic


def test_autotune_fp64_fft_choice_keeps_results():
    from paper_1604_05140_gb300 import Plan
    B, NB = 16, 3
    plan = Plan(B, NB, "fp64")
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 2)
    ct = torch.from_numpy(c).cuda()
    before = plan.forward(plan.inverse(ct)).cpu().numpy()
    jf, ji, rn, src = _parse(plan.autotune())
    assert src == "timed" and jf in (4, 8) and ji in (4, 8)
    after = plan.forward(plan.inverse(ct)).cpu().numpy()
    assert np.array_equal(before, after)  # ring grouping does not change the arithmetic


def test_autotune_rejects_host_buffers():
    from paper_1604_05140_gb300 import Plan, SGLError
    plan = Plan(8, 1, "fp64")
    with pytest.raises((SGLError, TypeError, ValueError)):
        plan.autotune(samples=torch.empty(plan.sample_shape, dtype=plan.dtype),
                      coeffs=torch.empty(plan.coeff_shape, dtype=plan.dtype))
