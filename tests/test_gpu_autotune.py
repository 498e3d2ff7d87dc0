"""Autotuner (sgl_autotune): timing-based choice of the launch configuration
(phi-FFT ring pairs per CTA, SIMT tile families, tensor-core tile widths),
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
    """(fft_fwd_jp, fft_inv_jp, rad_inv_narrow, source); the tile shapes are
    checked by _shapes."""
    m = re.match(r"fft_fwd_jp=(\d+) fft_inv_jp=(\d+) rad_inv_narrow=(\d+) simt=\d,\d,\d,\d rad_rows=\d+ "
                 r"fft_merge=[01] queue=[1248],[1248],[1248],[1248] inv_order=[01] source=(\w+)$", text)
    assert m, text
    return int(m.group(1)), int(m.group(2)), int(m.group(3)), m.group(4)


def _shapes(text):
    """(SIMT tile family of each GEMM stage, tensor-core radial tile width)."""
    m = re.search(r"simt=(\d),(\d),(\d),(\d) rad_rows=(\d+)", text)
    assert m, text
    return tuple(int(m.group(k)) for k in range(1, 5)), int(m.group(5))


def test_autotune_cache_and_parity(tmp_path):
    from paper_1604_05140_gb300 import Plan
    B, NB = 64, 4
    cache = str(tmp_path / "tuning.txt")
    plan = Plan(B, NB, "tf32x3")
    assert _parse(plan.tuning)[3] == "default"
    tuned = plan.autotune(cache=cache)
    jf, ji, rn, src = _parse(tuned)
    assert src == "timed" and jf in (4, 8, 16) and ji in (4, 8, 16) and rn in (1, 65)
    simt, rad_rows = _shapes(tuned)
    assert simt == (0, 0, 0, 0) and rad_rows in (32, 48, 64)  # tensor-core plan: the radial tile width
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
    cached = plan2.autotune(cache=cache)
    assert _parse(cached) == (jf, ji, rn, "cache") and _shapes(cached) == (simt, rad_rows)
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
    tuned = plan.autotune()
    jf, ji, rn, src = _parse(tuned)
    assert src == "timed" and jf in (4, 8) and ji in (4, 8)
    simt, _ = _shapes(tuned)
    assert all(p in (0, 1, 2) for p in simt)
    after = plan.forward(plan.inverse(ct)).cpu().numpy()
    # neither the ring grouping nor the SIMT tile family changes the
    # arithmetic: each output is one thread's sum over K in the same order
    assert np.array_equal(before, after)


def test_autotune_radial_tile_width_keeps_the_bound(tmp_path):
    # each tensor-core radial tile width the tuner may pick (forced through
    # the cache file): the round trip stays within the split-precision gate
    from paper_1604_05140_gb300 import Plan
    B, NB = 128, 1
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 8, decay=True)
    ct = torch.from_numpy(c).to(torch.complex64).cuda()
    first = str(tmp_path / "tuned.txt")
    Plan(B, NB, "tf32x3").autotune(cache=first)
    line = open(first).read().splitlines()[0]
    for rr in (32, 48, 64):
        forced = tmp_path / f"rr{rr}.txt"
        forced.write_text(re.sub(r"rad_rows=\d+", f"rad_rows={rr}", line) + "\n")
        plan = Plan(B, NB, "tf32x3")
        text = plan.autotune(cache=str(forced))
        assert _parse(text)[3] == "cache" and _shapes(text)[1] == rr, text
        f = plan.forward(plan.inverse(ct)).cpu().numpy()
        assert np.abs(f - c).max() / np.abs(c).max() < TF32X3_TOL, rr
        plan.check()


def test_merged_fft_launch_keeps_results(tmp_path):
    # an uneven plan runs its phi-FFT sizes in one multi-size launch per
    # direction (default) or one launch per size (forced through the cache):
    # each CTA runs the same code either way, so the results are identical
    from paper_1604_05140_gb300 import Plan
    Bs = [16, 24, 40, 56, 72, 128, 104]
    cs = [inputs.random_coeffs(b, 1, seed=1200 + k)[0] for k, b in enumerate(Bs)]
    ct = torch.from_numpy(np.concatenate(cs)).to(torch.complex64).cuda()
    merged = Plan.many(Bs, precision="tf32x3")
    f1 = merged.forward(merged.inverse(ct))
    first = str(tmp_path / "tuned.txt")
    Plan.many(Bs, precision="tf32x3").autotune(cache=first)
    line = open(first).read().splitlines()[0]
    # the default configuration, but for the merge choice
    line = re.sub(r"fft_fwd_jp=\d+ fft_inv_jp=\d+ rad_inv_narrow=\d+", "fft_fwd_jp=16 fft_inv_jp=16 rad_inv_narrow=65",
                  line)
    line = re.sub(r"rad_rows=\d+", "rad_rows=64", line)
    line = re.sub(r"queue=[\d,]+", "queue=2,2,2,2", line)
    line = re.sub(r"inv_order=\d", "inv_order=0", line)
    for fm in (0, 1):
        forced = tmp_path / f"fm{fm}.txt"
        forced.write_text(re.sub(r"fft_merge=\d", f"fft_merge={fm}", line) + "\n")
        plan = Plan.many(Bs, precision="tf32x3")
        text = plan.autotune(cache=str(forced))
        assert f"fft_merge={fm}" in text
        # seven FFT sizes: one launch per direction, or seven; two tensor-core stages
        assert plan.launches_per_call == (1 if fm else 7) + 2
        f2 = plan.forward(plan.inverse(ct))
        assert torch.equal(f1, f2), fm
        for k, b in enumerate(Bs):
            co = plan.coeff_offset(k)
            fk = f2[co:co + O.coeff_count(b)].cpu().numpy()
            assert np.abs(fk - cs[k]).max() / np.abs(cs[k]).max() < TF32X3_TOL, (fm, b)
        plan.check()


def test_work_queue_granularity_keeps_results(tmp_path):
    # the tensor-core stages take their tiles from a work queue of slices; the
    # number of slices per CTA and the inverse phi-FFT's CTA order (forced
    # through the cache) change which CTA runs a tile or a ring pair, never
    # its arithmetic: identical results
    from paper_1604_05140_gb300 import Plan
    Bs = [64, 16, 128, 40]
    cs = [inputs.random_coeffs(b, 1, seed=1300 + k)[0] for k, b in enumerate(Bs)]
    ct = torch.from_numpy(np.concatenate(cs)).to(torch.complex64).cuda()
    first = str(tmp_path / "tuned.txt")
    Plan.many(Bs, precision="tf32x3").autotune(cache=first)
    line = open(first).read().splitlines()[0]
    ref = None
    for q, io in (("1,1,1,1", 0), ("2,2,2,2", 1), ("4,8,1,2", 0), ("8,4,8,4", 1)):
        forced = tmp_path / f"q{q.replace(',', '')}_{io}.txt"
        forced.write_text(re.sub(r"inv_order=\d", f"inv_order={io}", re.sub(r"queue=[\d,]+", f"queue={q}", line)) + "\n")
        plan = Plan.many(Bs, precision="tf32x3")
        text = plan.autotune(cache=str(forced))
        assert f"queue={q}" in text and f"inv_order={io}" in text
        s = plan.inverse(ct)
        f = plan.forward(s)
        plan.check()
        if ref is None:
            ref = (s.clone(), f.clone())
        assert torch.equal(s, ref[0]) and torch.equal(f, ref[1]), q


def test_autotune_rejects_host_buffers():
    from paper_1604_05140_gb300 import Plan, SGLError
    plan = Plan(8, 1, "fp64")
    with pytest.raises((SGLError, TypeError, ValueError)):
        plan.autotune(samples=torch.empty(plan.sample_shape, dtype=plan.dtype),
                      coeffs=torch.empty(plan.coeff_shape, dtype=plan.dtype))
