"""Roofline bookkeeping of bench.py on the host (no GPU): which bound a
stage is measured against, the derived CUDA-core peaks, and the DRAM traffic
read from the committed ncu summaries only while the sources match them."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

STAGES = ("fft_forward", "legendre_forward", "radial_forward", "radial_inverse", "legendre_inverse", "fft_inverse")


def _stage(dominant, ms=10.0):
    return {k: ((ms if k == dominant else 1.0), 1) for k in STAGES}


def test_derived_alu_peaks():
    # 152 SMs x FMA lanes x 2 flops x 2.07 GHz; FP64 is GB300's nominal 1.25 TFLOP/s
    assert bench.alu_peak_tflops("fp64") == pytest.approx(1.25856)
    assert bench.alu_peak_tflops("fp32") == pytest.approx(80.548, rel=1e-4)


@pytest.mark.parametrize("prec,cbytes", [("fp64", 16), ("fp32", 8)])
def test_cuda_core_gemm_stage_is_alu_bound(prec, cbytes, monkeypatch):
    monkeypatch.setattr(bench, "BATCH", 4)
    r = bench.roofline(_stage("legendre_forward"), cbytes, prec)
    flops = bench.stage_model(bench.B_BENCH, 4, cbytes)["legendre_forward"][1]
    assert r["kernel"] == "legendre_forward" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / 10e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.alu_peak_tflops(prec))


@pytest.mark.parametrize("prec,dominant", [("fp64", "fft_inverse"), ("tf32x3", "legendre_forward"),
                                           ("tf32x3", "fft_inverse")])
def test_hbm_bound_otherwise(prec, dominant, monkeypatch):
    monkeypatch.setattr(bench, "BATCH", 4)
    cbytes = 16 if prec == "fp64" else 8
    r = bench.roofline(_stage(dominant), cbytes, prec)
    nbytes = bench.stage_model(bench.B_BENCH, 4, cbytes)[dominant][0]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(nbytes / 10e-3 / 1e9)


@pytest.mark.parametrize("prec,stage", [("tf32x3", "fft_inverse"), ("tf32x3", "legendre_forward"),
                                        ("fp64", "legendre_forward"), ("fp64", "radial_inverse")])
def test_traffic_only_for_matching_sources(prec, stage, monkeypatch):
    path = os.path.join(ROOT, "profiles", bench.TRAFFIC_PROFILES[prec])
    with open(path) as fh:
        recorded = [ln.split(":", 1)[1].strip() for ln in fh if ln.startswith("source-hash:")][0]
    monkeypatch.setattr(bench, "source_hash", lambda: recorded)
    per_fn = bench.measured_traffic(prec, stage, 1)
    assert per_fn > 0 and bench.measured_traffic(prec, stage, 64) == 64 * per_fn
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.measured_traffic(prec, stage, 64) is None
    assert bench.measured_traffic("bf16x3", stage, 64) is None


def test_tensor_core_stages_against_the_tensor_pipe(monkeypatch):
    # TF32x3: three TF32 products per useful multiply-add; streaming a
    # Legendre stage's bytes at the HBM peak bounds its tensor-pipe share at
    # 12 B^4 flops / (83.6 MB / HBM) / TF32 peak, independent of the batch
    monkeypatch.setattr(bench, "BATCH", 64)
    st = {k: (1.0, 1) for k in STAGES}
    r = bench.roofline(st, 8, "tf32x3")
    g = r["gemm_stages"]
    hbm, _ = bench.peaks()
    bf16, _ = bench.bf16_peak()
    B = bench.B_BENCH
    per_fn_bytes = 4 * B * B * (2 * B - 1) * 4 + 2 * B ** 3 * 4
    ceiling = 3 * 4 * B ** 4 / (per_fn_bytes / (hbm * 1e9)) / 1e12 / (bf16 / 2)
    assert g["legendre_forward"]["tensor_frac_at_hbm_peak"] == pytest.approx(ceiling)
    assert g["legendre_forward"]["mma_tflops"] == pytest.approx(3 * 4 * B ** 4 * 64 / 1e-3 / 1e12)
    assert set(g) >= set(bench.GEMM_STAGES)
    assert "gemm_stages" not in bench.roofline(st, 16, "fp64")


def test_round_trip_error_metrics():
    # the three error measures of the bench line on a hand-made case: two
    # functions, the second with one coefficient off by 1e-6 of the largest
    torch = pytest.importorskip("torch")
    c = torch.tensor([[1.0 + 0j, 0.5j, -0.25], [2.0, 1.0j, 1e-3]], dtype=torch.complex128)
    c2 = c.clone()
    c2[1, 2] += 2e-6
    e = bench.error_metrics(c, c2)
    assert e["normwise_max"] == pytest.approx(2e-6 / 2.0)
    assert e["l2"] == pytest.approx(2e-6 / (4 + 1 + 1e-6) ** 0.5)
    assert e["per_coefficient"] == pytest.approx(2e-6 / 1e-3)
    assert bench.error_metrics(c, c.clone()) == {"normwise_max": 0.0, "l2": 0.0, "per_coefficient": 0.0}


def test_cores_used_is_cpu_time_over_wall_time():
    assert bench.cores_used(10.0, 10.2) == 1
    assert bench.cores_used(10.0, 0.5) == 1
    assert bench.cores_used(2.0, 7.9) == 4
    assert bench.cores_used(0.0, 1.0) == 1


def test_cpu_oracle_sample_line():
    r = bench.cpu_oracle_sample(B=8, budget_s=0.2)
    assert r["kind"] == "oracle" and r["unit"] == "transforms/s" and r["value"] > 0
    assert 1 <= r["cores"] <= r["threads_available"] and r["cpu_s"] > 0
    assert "B=8" in r["sample"]


def test_error_gate_names_every_missed_bound():
    # the bench exits non-zero when a round trip misses its bound: 1e-12
    # normwise for FP64, 1e-6 for the split-precision paths; the reduced
    # precision variants (TF32 hi*hi, BF16x3) have no such bound
    ok = {"config": {"precision": "tf32x3"}, "round_trip_errors": {"normwise_max": 8e-7},
          "fp64_path": {"round_trip_errors": {"normwise_max": 5e-15}},
          "variants": {"fp16x3": {"round_trip_errors": {"normwise_max": 7e-7}, "round_trip_max_rel_err": 6e-7},
                       "bf16x3": {"round_trip_errors": {"normwise_max": 7e-6}, "round_trip_max_rel_err": 7e-6}}}
    assert bench.error_gate(ok) == []
    bad = {"config": {"precision": "tf32x3"}, "round_trip_errors": {"normwise_max": 1.5e-6},
           "fp64_path": {"round_trip_errors": {"normwise_max": 2e-12}},
           "variants": {"fp16x3": {"round_trip_errors": {"normwise_max": 3e-6}, "round_trip_max_rel_err": 9e-7}}}
    missed = bench.error_gate(bad)
    assert len(missed) == 3
    assert any(m.startswith("tf32x3") for m in missed) and any(m.startswith("fp64") for m in missed)
    assert any(m.startswith("fp16x3") for m in missed)
