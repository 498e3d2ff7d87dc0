"""Benchmark: SGL inverse + forward transform throughput at B=128, batch 64.

One step = one sgl_inverse followed by one sgl_forward over a batch of 64
functions of bandlimit B=128 (coefficients complex normal with 1/n decay,
seeded; the paper's experiment of Sect. 4 run as a batch).  The headline
line is the split-precision path (TF32x3 tensor-core stages); the plain FP64
GPU path is timed on the same workload and reported alongside.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs an independent replica of the batch (the
transform of one function never needs another function's data), so the job
scales weakly with no data-path collective; `--gpus N` outside a launcher
starts the N ranks itself.  The exit status is 3 when the round trip misses
its error bound (1e-12 FP64, 1e-6 split precision), after the line is printed.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SGL fwd+inv transforms/sec and coeffs/sec at B=128, FP64 vs split-precision"
B_BENCH = 128
TUNE = True
BATCH = 64
L2_BYTES = 129 * 1024 * 1024


def omega_count(B):
    return B * (B + 1) * (2 * B + 1) // 6


# CUDA-core arithmetic peak of GB300: 152 SMs at the 2070 MHz maximum SM
# clock; FMA lanes per SM per clock: 128 in FP32, 2 in FP64 (152 x 2 x 2 flops
# x 2.07 GHz = 1.26 TFLOP/s, the nominal FP64 rate).  FP64 and FP32 plans run
# their Legendre and radial stages as GEMMs on these units.
SMS = 152
SM_MAX_MHZ = 2070
SIMT_FMA_LANES = {"fp32": 128, "fp64": 2}
GEMM_STAGES = ("legendre_forward", "radial_forward", "radial_inverse", "legendre_inverse")


def alu_peak_tflops(prec):
    return SMS * SIMT_FMA_LANES[prec] * 2 * SM_MAX_MHZ * 1e6 / 1e12


# tensor-core precisions: MMA products per useful multiply-add and the dense
# peak of their operand type relative to bf16 (TF32 runs at half the rate)
TC_PRECS = {"tf32x3": (3, 0.5), "tf32": (1, 0.5), "bf16x3": (3, 1.0), "fp16x3": (3, 1.0)}


def bf16_peak():
    """Measured dense bf16 TF/s (burst: each stage is timed as one launch
    inside a short step, below the power cap), else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        if "bf16_tflops" in d:
            return d["bf16_tflops"], "measured"
    return 1900.0, "fallback"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes / flops per launch of each stage (whole batch)
# ---------------------------------------------------------------------------

def stage_model(B, NB, cbytes):
    """Bytes each stage must move (its inputs and outputs, once) and flops.

    cbytes: bytes of one complex element (16 FP64, 8 FP32).  Real element
    rb = cbytes/2.  Per function: samples 4B^3 complex, coefficients Omega
    complex, E/O (or G) spectra 4B^2(2B-1) reals, S spectra 2B^3 reals.
    """
    rb = cbytes // 2
    samp = 4 * B ** 3 * cbytes
    coef = omega_count(B) * cbytes
    w1 = 4 * B * B * (2 * B - 1) * rb
    w2 = 2 * B ** 3 * rb
    n = 2 * B
    fft_flops = B * (2 * B) * 5 * n * np.log2(n)  # B*2B rings, 5 N log2 N each
    leg_flops = 0
    for m in range(-(B - 1), B):
        am = abs(m)
        leg_flops += 2 * (B - am) * B * (2 * B)  # (B-|m|) rows, K=B (folded), 2B real columns (re,im of B shells)
    rad_flops = 2 * 2 * B * omega_count(B)       # per coefficient: B-term complex x real sum
    return {
        "fft_forward": (NB * (samp + w1), NB * fft_flops),
        "legendre_forward": (NB * (w1 + w2), NB * leg_flops),
        "radial_forward": (NB * (w2 + coef), NB * rad_flops),
        "radial_inverse": (NB * (coef + w2), NB * rad_flops),
        "legendre_inverse": (NB * (w2 + w1), NB * leg_flops),
        "fft_inverse": (NB * (w1 + samp), NB * fft_flops),
    }


# ---------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # wait for the first sample, then keep only samples taken from now on
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smmax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "first", 0):]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smmax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smmax) if smmax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# distributed helpers (replicas)
# ---------------------------------------------------------------------------

def dist_setup():
    """One process per GPU (replicas): NCCL when CUDA is present, else gloo
    (host-only runs of the replica logic)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            backend = "nccl"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x):
    """Maximum of x over the ranks."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(ws, batch, ms_local):
    """Whole-job throughput of `ws` replicas that each transformed `batch`
    functions: all functions over the slowest rank's time.  Returns
    (transforms/s, ms of the slowest rank)."""
    ms = allmax(ws, ms_local)
    return ws * batch / (ms * 1e-3), ms


# ---------------------------------------------------------------------------
# CPU baseline: the oracle
# ---------------------------------------------------------------------------

def cores_used(wall_s, cpu_s):
    """Threads the oracle kept busy on average: process CPU time over wall
    time (the oracle's NumPy work is mostly single-threaded whatever the size
    of the BLAS pool)."""
    return max(1, round(cpu_s / wall_s)) if wall_s > 0 else 1


def _oracle_serve(B, inq, outq):
    """Worker process of OraclePool: builds the oracle's tables, then runs one
    whole function (inverse, then forward) per seed it receives and returns
    the CPU seconds it took; None ends it."""
    import oracle as O
    from paper_1604_05140_gb300 import inputs
    O.legendre_table(B)
    O.radial_table(B)  # tables are set-up, not part of a transform
    outq.put("ready")
    while True:
        seed = inq.get()
        if seed is None:
            return
        p0 = time.process_time()
        c = inputs.random_coeffs(B, 1, seed=seed, decay=True)
        O.forward(O.inverse(c, B), B)
        outq.put(time.process_time() - p0)


class OraclePool:
    """`workers` processes (spawned, so that none inherits a CUDA context; one
    BLAS thread each) that transform whole functions of the workload with the
    FP64 oracle in parallel: the oracle as it stands, on the host's cores."""

    BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __init__(self, workers, B=B_BENCH):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in self.BLAS_ENV}
        for k in self.BLAS_ENV:
            os.environ[k] = "1"
        try:
            self.inq = [ctx.Queue() for _ in range(workers)]
            self.outq = ctx.Queue()
            self.procs = [ctx.Process(target=_oracle_serve, args=(B, q, self.outq), daemon=True) for q in self.inq]
            for p in self.procs:
                p.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for _ in self.procs:
            self.outq.get()
        self.workers = workers

    def run(self, seed0):
        """One function per worker (seeds seed0, seed0 + 1, ...); returns the
        wall seconds until the last finished and the summed CPU seconds."""
        t0 = time.perf_counter()
        for k, q in enumerate(self.inq):
            q.put(seed0 + k)
        cpu = sum(self.outq.get() for _ in self.inq)
        return time.perf_counter() - t0, cpu

    def close(self):
        for q in self.inq:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)


def host_workers():
    """Oracle worker processes for the all-cores baseline: one per host core."""
    return os.cpu_count() or 1


def cpu_oracle_sample(B=B_BENCH, budget_s=12.0, seed=1604051403, workers=None):
    """Times the FP64 oracle (inverse then forward) on whole functions of the
    benchmark workload, on one core and on all host cores (one process per
    core), each for about budget_s / 2 seconds."""
    workers = workers or host_workers()
    out = {}
    for key, w in (("all", workers), ("one", 1)):
        pool = OraclePool(w, B)
        n, wall, cpu = 0, 0.0, 0.0
        while wall < budget_s / 2:
            dt, c = pool.run(seed + n)
            n, wall, cpu = n + w, wall + dt, cpu + c
        pool.close()
        out[key] = (n, wall, cpu, w)
    n, wall, cpu, w = out["all"]
    n1, wall1, cpu1, _ = out["one"]
    return {"value": n / wall, "unit": "transforms/s", "cores": w, "kind": "oracle",
            "threads_available": os.cpu_count(), "cpu_s": cpu,
            "sample": f"{n} whole functions of B={B} (inverse + forward each, {w} at a time in {w} processes "
                      f"of one BLAS thread) out of the batch of {BATCH}, {wall:.1f} s, FP64 NumPy separated form",
            "one_thread": {"value": n1 / wall1, "unit": "transforms/s", "cores": 1, "cpu_s": cpu1,
                           "sample": f"{n1} whole functions of B={B} in one process, {wall1:.1f} s"}}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_path(precision, steps, warmup, ws, rank, profile=True):
    import torch
    from paper_1604_05140_gb300 import Plan, inputs, sgl

    plan = Plan(B_BENCH, BATCH, precision)
    if TUNE:
        plan.autotune()  # launch configuration chosen by timing (setup, not timed)
    lib = sgl.load_library()
    c_np = inputs.random_coeffs(B_BENCH, BATCH, seed=inputs.BASE_SEED + 3 + 1000 * rank, decay=True)
    c = torch.from_numpy(c_np).to(plan.dtype).cuda()
    s = torch.empty(plan.sample_shape, dtype=plan.dtype, device="cuda")
    c2 = torch.empty(plan.coeff_shape, dtype=plan.dtype, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.inverse(c, out=s)
        plan.forward(s, out=c2)
    torch.cuda.synchronize()
    err = float((c2 - c).abs().max().item() / c.abs().max().item())
    barrier(ws)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        # per-stage events from the second step on: the first stage after the
        # synchronize would also hold the host's latency to its first launch
        if profile and k == min(1, steps - 1):
            lib.sgl_set_profiling(plan.handle, 1)
        plan.inverse(c, out=s)
        plan.forward(s, out=c2)
    ev1.record(stream)
    torch.cuda.synchronize()
    plan.check()  # raises if any bounded device-side wait gave up during the run
    barrier(ws)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / steps
    stage = {}
    if profile:
        import ctypes
        n = 6
        tms = (ctypes.c_double * n)()
        tl = (ctypes.c_int64 * n)()
        lib.sgl_stage_times(plan.handle, tms, tl)
        for k in range(n):
            if tl[k]:
                stage[lib.sgl_stage_name(k).decode()] = (tms[k] / tl[k], int(tl[k]))
        lib.sgl_set_profiling(plan.handle, 0)
    launches = plan.launches_per_call * 2 * steps
    return plan, ms, stage, clocks, err, launches, (c_np, c, s, c2)


def real_path(steps, warmup):
    """Real functions: 64 real functions of B=128 in one TF32x3 plan of real
    functions (two per complex transform, separated by the coefficient
    symmetry of real functions).  Round trip on coefficients of real
    functions (the symmetric part of random decaying coefficients, obtained
    by one round trip), timed with CUDA events like the main workload."""
    import torch
    from paper_1604_05140_gb300 import Plan, inputs
    plan = Plan(B_BENCH, BATCH, "tf32x3", samples="real")
    if TUNE:
        plan.autotune()
    c0 = torch.from_numpy(inputs.random_coeffs(B_BENCH, BATCH, seed=inputs.BASE_SEED + 5, decay=True)).to(
        torch.complex64).cuda()
    s = torch.empty(plan.sample_shape, dtype=plan.sample_dtype, device="cuda")
    c = torch.empty(plan.coeff_shape, dtype=plan.dtype, device="cuda")
    c2 = torch.empty_like(c)
    plan.inverse(c0, out=s)
    plan.forward(s, out=c)  # coefficients of real functions
    for _ in range(max(1, warmup)):
        plan.inverse(c, out=s)
        plan.forward(s, out=c2)
    torch.cuda.synchronize()
    err = float((c2 - c).abs().max().item() / c.abs().max().item())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        plan.inverse(c, out=s)
        plan.forward(s, out=c2)
    ev1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = ev0.elapsed_time(ev1) / steps
    return {"workload": f"{BATCH} real functions, B={B_BENCH}, TF32x3, two per complex transform",
            "value": BATCH / (ms * 1e-3), "unit": "transforms/s", "ms_per_step": ms, "steps": steps,
            "round_trip_max_rel_err": err, "launches_per_round_trip": 2 * plan.launches_per_call,
            "sample_bytes_per_function": 4 * B_BENCH ** 3 * 4}


def paper_grid_path(steps, warmup):
    """The paper's own grid (2B half-range Gauss-Hermite radii): the paper's
    timing configuration (B=64, one function, round trip in FP64, as in its
    Table 2) and B=128 x 16 functions in FP64, FP32 and TF32x3 (the
    tensor-core stages run each function's radii as two halves), and 16 real
    functions in TF32x3 (paired, then halved).  Round trip on seeded decaying
    coefficients (real functions: on the coefficients of the real part of
    their inverse, which the round trip reproduces), CUDA events."""
    import torch
    from paper_1604_05140_gb300 import Plan, inputs
    out = {}
    for label, B, nb, prec, samples in (("b64x1_fp64", 64, 1, "fp64", "weighted"),
                                        ("b128x16_fp64", 128, 16, "fp64", "weighted"),
                                        ("b128x16_fp32", 128, 16, "fp32", "weighted"),
                                        ("b128x16_tf32x3", 128, 16, "tf32x3", "weighted"),
                                        ("b128x16_tf32x3_real", 128, 16, "tf32x3", "real")):
        plan = Plan(B, nb, prec, samples=samples, grid="hermite")
        c = torch.from_numpy(inputs.random_coeffs(B, nb, seed=inputs.BASE_SEED + 6, decay=True)).to(plan.dtype).cuda()
        s = torch.empty(plan.sample_shape, dtype=plan.sample_dtype, device="cuda")
        c2 = torch.empty_like(c)
        if samples == "real":
            plan.inverse(c, out=s)
            plan.forward(s, out=c2)
            c = c2.clone()
        for _ in range(max(1, warmup)):
            plan.inverse(c, out=s)
            plan.forward(s, out=c2)
        torch.cuda.synchronize()
        err = float((c2 - c).abs().max().item() / c.abs().max().item())
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            plan.inverse(c, out=s)
            plan.forward(s, out=c2)
        ev1.record()
        torch.cuda.synchronize()
        plan.check()
        ms = ev0.elapsed_time(ev1) / steps
        out[label] = {"B": B, "batch": nb, "precision": prec, "samples": samples, "radii": 2 * B, "ms_per_step": ms,
                      "value": nb / (ms * 1e-3), "unit": "transforms/s", "steps": steps,
                      "round_trip_max_rel_err": err}
        del plan, s, c, c2
    return out


def midpoint_path(reps=3):
    """Accuracy and cost of the Cartesian midpoint rule (sgl_midpoint, the
    practice of the paper's Discussion) against the SGL transform, FP64, on 16
    random complex polynomials of degree <= 3 (band-limited: the SGL sampling
    theorem makes the transform exact, so its coefficients are the reference).
    B = 16, cube [-6, 6]^3, M = 24 .. 64 cells per axis."""
    import torch
    from paper_1604_05140_gb300 import Plan, midpoint
    B, nf, L = 16, 16, 6.0
    rng = np.random.default_rng(1604051407)
    mons = [(i, j, k) for i in range(4) for j in range(4) for k in range(4) if i + j + k <= 3]
    cf = rng.standard_normal((nf, len(mons))) + 1j * rng.standard_normal((nf, len(mons)))

    def sample(x, y, z):
        return np.stack([sum(c * x ** i * y ** j * z ** k for c, (i, j, k) in zip(cf[q], mons)) for q in range(nf)])

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    plan = Plan(B, nf, "fp64", samples="physical")
    r, th, ph, _, _ = plan.grid()
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    fs = torch.from_numpy(sample(R * np.sin(TH) * np.cos(PH), R * np.sin(TH) * np.sin(PH), R * np.cos(TH))).cuda()
    ref, ms = timed(lambda: plan.forward(fs))
    ref = ref.cpu().numpy()
    res = {"B": B, "functions": nf, "cube_half_width": L, "reference": "the SGL transform (exact for these functions)",
           "sgl": {"ms": ms, "samples_per_function": 4 * B ** 3}, "midpoint": {}}
    for M in (24, 32, 48, 64):
        x, y, z, _ = cartesian_midpoints(M, L)
        fm = torch.from_numpy(sample(x, y, z)).cuda()
        got, ms = timed(lambda: midpoint(fm, B, L))
        err = float(np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max())
        # roofline: the FP64 pipe; algorithmic work 8 flops (one complex
        # multiply-add of f by the conjugated basis value) per point,
        # coefficient and function (the per-point basis tables not counted)
        fl = 8.0 * M ** 3 * omega_count(B) * nf
        tf = fl / (ms * 1e-3) / 1e12
        res["midpoint"][str(M)] = {"ms": ms, "samples_per_function": M ** 3, "max_rel_err": err,
                                   "roofline": {"bound": "alu", "achieved": tf, "peak": alu_peak_tflops("fp64"),
                                                "unit": "TFLOP/s", "frac": tf / alu_peak_tflops("fp64"),
                                                "algorithmic_flops": fl,
                                                "peak_source": "derived: FP64 FMA lanes x clock"}}
        del fm
    return res


def cartesian_midpoints(M, L):
    """Cell midpoints of [-L, L]^3 (the grid sgl_midpoint samples on)."""
    h = 2.0 * L / M
    c = -L + (np.arange(M) + 0.5) * h
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z, h ** 3


def seminaive_path(steps=3, warmup=1):
    """The forward transform with direct and with seminaive Legendre sums
    (sgl_set_dlt), FP64, B = 128 x 64: forward time and Legendre stage time
    (per-stage CUDA events)."""
    import ctypes
    import torch
    from paper_1604_05140_gb300 import Plan, inputs, sgl
    lib = sgl.load_library()
    plan = Plan(B_BENCH, BATCH, "fp64")
    c = torch.from_numpy(inputs.random_coeffs(B_BENCH, BATCH, seed=inputs.BASE_SEED + 3, decay=True)).cuda()
    s = plan.inverse(c)
    out = {"B": B_BENCH, "batch": BATCH, "precision": "fp64"}
    for label, on in (("direct", False), ("seminaive", True)):
        plan.set_dlt(on)
        f = torch.empty_like(c)
        for _ in range(max(1, warmup)):
            plan.forward(s, out=f)
        torch.cuda.synchronize()
        err = float((f - c).abs().max().item() / c.abs().max().item())
        lib.sgl_set_profiling(plan.handle, 1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            plan.forward(s, out=f)
        ev1.record()
        torch.cuda.synchronize()
        tms = (ctypes.c_double * 6)()
        tl = (ctypes.c_int64 * 6)()
        lib.sgl_stage_times(plan.handle, tms, tl)
        lib.sgl_set_profiling(plan.handle, 0)
        out[label] = {"forward_ms": ev0.elapsed_time(ev1) / steps, "legendre_forward_ms": tms[1] / max(tl[1], 1),
                      "max_rel_err": err}
    plan.check()
    return out


def uneven_path(steps, warmup):
    """The batching workload: 256 functions with bandlimits uniform in
    {16, 24, ..., 128} in one TF32x3 plan; each call of the round trip is one
    launch of the plan's own CUDA graph (sgl_set_graphs: the plan captures its
    launches once per direction and buffer pair); per-function error against
    the input coefficients."""
    import torch
    from paper_1604_05140_gb300 import Plan, inputs
    Bs = [int(b) for b in inputs.uneven_bandlimits(256)]
    plan = Plan.many(Bs, precision="tf32x3")
    if TUNE:
        plan.autotune()
    plan.set_graphs(True)
    cs = [inputs.random_coeffs(B, 1, seed=inputs.BASE_SEED + 4 + 10 * k)[0] for k, B in enumerate(Bs)]
    c = torch.from_numpy(np.concatenate(cs)).to(torch.complex64).cuda()
    s = torch.empty(plan.sample_shape, dtype=plan.dtype, device="cuda")
    out = torch.empty(plan.coeff_shape, dtype=plan.dtype, device="cuda")
    for _ in range(max(1, warmup)):  # the first round trip captures the two graphs
        plan.inverse(c, out=s)
        plan.forward(s, out=out)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        plan.inverse(c, out=s)
        plan.forward(s, out=out)
    ev1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = ev0.elapsed_time(ev1) / steps
    f = out.cpu().numpy()
    err = 0.0
    for k, B in enumerate(Bs):
        co = plan.coeff_offset(k)
        fk = f[co:co + len(cs[k])]
        err = max(err, float(np.abs(fk - cs[k]).max() / np.abs(cs[k]).max()))
    return {"workload": "256 functions, B uniform in {16, 24, ..., 128}, TF32x3, the plan's own CUDA graph per call",
            "value": len(Bs) / (ms * 1e-3), "unit": "transforms/s", "ms_per_step": ms, "steps": steps,
            "segments": len(set(Bs)), "launches_per_round_trip": 2 * plan.launches_per_call,
            "graph_launches_per_round_trip": 2, "graphs": plan.graph_count,
            "max_rel_err": err, "launch_config": plan.tuning}


def profile_case(case, precision, steps, warmup):
    """Round trips of one workload and nothing else, for profiler captures
    (`--profile-case`): the uneven-bandlimit batch (256 functions, B in
    {16, ..., 128}), the uniform one (B = 128, --batch functions), the same on
    the paper's grid, or the midpoint rule (B = 16, M = 32, 16 functions);
    eager launches, default launch configuration.  Prints one JSON line with
    the mean step time; not a benchmark line."""
    import torch
    from paper_1604_05140_gb300 import Plan, inputs, midpoint
    if case == "midpoint":  # the midpoint rule, B = 16, M = 32, 16 functions, FP64
        fm = torch.from_numpy(inputs.random_samples(1, 16 * 32 ** 3 // 4, seed=inputs.BASE_SEED + 9)
                              .reshape(16, 32, 32, 32)).cuda()
        for _ in range(warmup + steps):
            midpoint(fm, 16, 6.0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": case, "steps": steps, "warmup": warmup}), flush=True)
        return
    if case == "uneven":
        Bs = [int(b) for b in inputs.uneven_bandlimits(256)]
        plan = Plan.many(Bs, precision=precision)
        c = np.concatenate([inputs.random_coeffs(B, 1, seed=inputs.BASE_SEED + 4 + 10 * k)[0]
                            for k, B in enumerate(Bs)])
    elif case == "paper_grid":  # the paper's 2B half-range Gauss-Hermite radii
        plan = Plan(B_BENCH, BATCH, precision, grid="hermite")
        c = inputs.random_coeffs(B_BENCH, BATCH, seed=inputs.BASE_SEED + 3, decay=True)
    else:
        plan = Plan(B_BENCH, BATCH, precision)
        c = inputs.random_coeffs(B_BENCH, BATCH, seed=inputs.BASE_SEED + 3, decay=True)
    c = torch.from_numpy(c).to(plan.dtype).cuda()
    s = torch.empty(plan.sample_shape, dtype=plan.dtype, device="cuda")
    out = torch.empty(plan.coeff_shape, dtype=plan.dtype, device="cuda")
    for _ in range(warmup):
        plan.inverse(c, out=s)
        plan.forward(s, out=out)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        plan.inverse(c, out=s)
        plan.forward(s, out=out)
    ev1.record()
    torch.cuda.synchronize()
    plan.check()
    print(json.dumps({"profile_case": case, "precision": precision, "steps": steps, "warmup": warmup,
                      "ms_per_step": ev0.elapsed_time(ev1) / steps,
                      "launches_per_round_trip": 2 * plan.launches_per_call}), flush=True)


def error_metrics(c, c2):
    """Round-trip errors of the coefficients c2 = forward(inverse(c)) against c,
    both (batch, Omega) tensors: the normwise max|d| / max|c| per function (the
    tests' gate), the per-function l2 ratio ||d|| / ||c||, and the paper's
    per-coefficient max |d_w| / |c_w| (Sect. 4), each the worst function."""
    d = (c2 - c).abs().double()
    a = c.abs().double()
    return {"normwise_max": float((d.amax(dim=1) / a.amax(dim=1)).max()),
            "l2": float((d.norm(dim=1) / a.norm(dim=1)).max()),
            "per_coefficient": float((d / a).max())}


def e2e_path(plan, c_np, steps, warmup, windows=3):
    """Same step through the C ABI with host buffers: pinned host coefficients
    in, pinned host coefficients out; the library stages the copies.  Timed
    on the host clock in `windows` windows of `steps` steps (the host link is
    shared with the machine's other work); returns the median window's time
    per step, every window's time per step (ms) and the bytes per copy."""
    import torch
    c_host = torch.from_numpy(c_np).to(plan.dtype).pin_memory()
    out_host = torch.empty(plan.coeff_shape, dtype=plan.dtype).pin_memory()
    s = torch.empty(plan.sample_shape, dtype=plan.dtype, device="cuda")
    for _ in range(max(1, warmup)):
        plan.inverse(c_host, out=s)
        plan.forward(s, out=out_host)
    torch.cuda.synchronize()
    per_step = []
    for _ in range(windows):
        t0 = time.perf_counter()
        for _ in range(steps):
            plan.inverse(c_host, out=s)
            plan.forward(s, out=out_host)
        torch.cuda.synchronize()
        per_step.append((time.perf_counter() - t0) / steps)
    nbytes = c_host.numel() * c_host.element_size()
    return sorted(per_step)[len(per_step) // 2], [t * 1e3 for t in per_step], nbytes


# the sources of the transform's stage kernels and their launch schedules
# (the midpoint rule, the no-allocation entry point, the self-test and the
# host-side quadrature tables do not change a stage kernel's traffic)
STAGE_SOURCES = ("api.cu", "fft16.cu", "kernels.cu", "sgl_internal.h", "tc_gemm.cu", "tc_inv.cu", "tc_ptx.cuh")


def source_hash():
    """Hash of the stage kernels' sources (names and contents)."""
    import hashlib
    h = hashlib.sha256()
    for name in STAGE_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_1604_05140_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TRAFFIC_PROFILES = {"tf32x3": "tf32x3_kernels_b128x4_dram.md", "fp64": "fp64_simt_gemm_b128x2.md"}


def measured_traffic(prec, kernel, batch):
    """DRAM bytes of one stage of `kernel` from the committed ncu capture
    (per function x batch), or None when the capture is for other sources."""
    if prec not in TRAFFIC_PROFILES:
        return None
    path = os.path.join(ROOT, "profiles", TRAFFIC_PROFILES[prec])
    if not os.path.exists(path):
        return None
    recorded, per_fn = None, {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("source-hash:"):
                recorded = line.split(":", 1)[1].strip()
            if line.startswith("dram-bytes-per-function:"):
                for kv in line.split(":", 1)[1].split():
                    k, v = kv.split("=")
                    per_fn[k] = int(v)
    if recorded != source_hash() or kernel not in per_fn:
        return None
    return per_fn[kernel] * batch


def roofline(stage, cbytes, prec):
    hbm, src = peaks()
    model = stage_model(B_BENCH, BATCH, cbytes)
    dom = max(stage, key=lambda k: stage[k][0] * stage[k][1])
    ms, nl = stage[dom]
    nbytes, flops = model[dom]
    out = {"kernel": dom, "bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
           "traffic": measured_traffic(prec, dom, BATCH), "peak_source": src, "launch_ms": ms,
           "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
           "stage_ms": {k: v[0] for k, v in stage.items()}}
    if prec in SIMT_FMA_LANES and dom in GEMM_STAGES:
        # a GEMM on the CUDA cores: bound by the FMA pipe of its precision
        out.update(bound="alu", achieved=flops / (ms * 1e-3) / 1e12, peak=alu_peak_tflops(prec), unit="TFLOP/s",
                   peak_source=f"derived: {SMS} SMs x {SIMT_FMA_LANES[prec]} {prec.upper()} FMA/clk x 2 flops"
                               f" x {SM_MAX_MHZ} MHz")
    out["frac"] = out["achieved"] / out["peak"]
    if prec in TC_PRECS:
        # the tcgen05 GEMM stages against the tensor pipe: achieved MMA rate,
        # and the most that streaming their bytes at the HBM peak would allow
        nprod, ratio = TC_PRECS[prec]
        bf16, bsrc = bf16_peak()
        tpeak = bf16 * ratio
        out["gemm_stages"] = {"tensor_peak_tflops": tpeak, "tensor_peak_source": f"{bsrc} bf16 x {ratio}"}
        for k in GEMM_STAGES:
            if k not in stage:
                continue
            nb, fl = model[k]
            t = stage[k][0] * 1e-3
            out["gemm_stages"][k] = {
                "mma_tflops": nprod * fl / t / 1e12,
                "frac_tensor_peak": nprod * fl / t / 1e12 / tpeak,
                "tensor_frac_at_hbm_peak": nprod * fl / (nb / (hbm * 1e9)) / 1e12 / tpeak,
                "frac_hbm": nb / t / 1e9 / hbm,
            }
    return out


def run_ours(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if not torch.cuda.is_available() or ws > torch.cuda.device_count():
        print(f"bench.py: {ws} rank(s) need as many visible GPUs; found "
              f"{torch.cuda.device_count() if torch.cuda.is_available() else 0}", file=sys.stderr)
        sys.exit(2)
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    precs = [args.precision] + ([] if args.no_fp64 or args.precision == "fp64" else ["fp64"])
    results = {}
    for prec in precs:
        steps = args.steps if prec != "fp64" else max(1, min(args.steps, args.fp64_steps))
        plan, ms, stage, clocks, err, launches, bufs = time_path(prec, steps, args.warmup, ws, rank)
        value_p, ms_max = whole_job(ws, BATCH, ms)
        results[prec] = dict(plan=plan, ms=ms_max, value=value_p, stage=stage, clocks=clocks, err=err,
                             launches=launches, steps=steps, bufs=bufs)
    head = results[args.precision]
    plan = head["plan"]
    cbytes = 16 if args.precision == "fp64" else 8
    value = head["value"]
    rl = roofline(head["stage"], cbytes, args.precision)
    # warm-up as for the device-buffer steps, at least 5 round trips: the first
    # host-buffer calls on freshly pinned buffers run slower (measured 27, 15,
    # then 7 ms per step in consecutive 5-step windows after 2 warm-up steps)
    e2e_dt, e2e_windows, nbytes = e2e_path(plan, head["bufs"][0], max(3, min(args.steps, 10)), max(5, args.warmup))
    e2e_value, _ = whole_job(ws, BATCH, e2e_dt * 1e3)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "transforms/s",
        "n_gpus": ws,
        "steps": head["steps"],
        "warmup": args.warmup,
        "ms_per_step": head["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "tf32x3": "tf32x3+f32acc", "tf32": "tf32+f32acc",
                  "bf16x3": "bf16x3+f32acc", "fp16x3": "fp16x3+f32acc"}[args.precision],
        "data": "synthetic: seeded complex-normal SGL coefficients with 1/n decay, synthesized to samples by the inverse",
        "config": {"workload": f"SGL inverse+forward, B={B_BENCH}, batch {BATCH} functions per GPU",
                   "B": B_BENCH, "batch": BATCH, "precision": args.precision,
                   "samples_bytes_per_function": 4 * B_BENCH ** 3 * cbytes,
                   "l2": "inputs larger than L2 (samples 4.3 GB per batch in FP32, 8.6 GB in FP64)",
                   "parallelism": f"replicas x{ws}", "launch_config": plan.tuning},
        "coeffs_per_s": value * omega_count(B_BENCH),
        "round_trip_max_rel_err": head["err"],
        "round_trip_errors": error_metrics(head["bufs"][1], head["bufs"][3]),
        "roofline": rl,
        "e2e": {"value": e2e_value, "unit": "transforms/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "window_ms_per_step": e2e_windows, "statistic": "median of the windows"},
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
    }
    if not args.no_variants and args.precision == "tf32x3":
        # reduced-precision variant of the tensor-core stages, same workload
        line["variants"] = {}
        for vp in ("fp16x3", "tf32", "bf16x3"):
            v_plan, v_ms, v_stage, v_clocks, v_err, _, v_bufs = time_path(vp, args.steps, args.warmup, ws, rank)
            v_value, v_ms = whole_job(ws, BATCH, v_ms)
            line["variants"][vp] = {"value": v_value, "unit": "transforms/s", "ms_per_step": v_ms,
                                    "round_trip_max_rel_err": v_err,
                                    "round_trip_errors": error_metrics(v_bufs[1], v_bufs[3]),
                                    "stage_ms": {k: v[0] for k, v in v_stage.items()}}
            del v_plan, v_bufs
    if not args.no_variants and args.precision == "tf32x3" and ws == 1:
        line["uneven_batch"] = uneven_path(max(3, min(args.steps, 20)), args.warmup)
        line["real_functions"] = real_path(max(3, min(args.steps, 20)), args.warmup)
        line["paper_grid"] = paper_grid_path(3, 1)
        line["midpoint_comparison"] = midpoint_path()
        line["seminaive_dlt"] = seminaive_path()
    if "fp64" in results and args.precision != "fp64":
        r = results["fp64"]
        line["fp64_path"] = {"value": r["value"], "unit": "transforms/s", "ms_per_step": r["ms"],
                             "steps": r["steps"], "round_trip_max_rel_err": r["err"],
                             "round_trip_errors": error_metrics(r["bufs"][1], r["bufs"][3]),
                             "stage_ms": {k: v[0] for k, v in r["stage"].items()}, "clocks": r["clocks"],
                             "roofline": roofline(r["stage"], 16, "fp64")}
        line["split_vs_fp64"] = line["value"] / line["fp64_path"]["value"]
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample(budget_s=args.cpu_seconds, workers=args.cpu_workers)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    missed = error_gate(line)
    if missed:
        print("bench.py: error bound missed: " + "; ".join(missed), file=sys.stderr)
        sys.exit(3)


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step: one whole function of the workload (inverse + forward) per
    # host core, in parallel worker processes running the oracle
    workers = args.cpu_workers or host_workers()
    pool = OraclePool(workers, B_BENCH)
    for w in range(args.warmup):
        pool.run(7 + w * workers)
    times, cpu = [], 0.0
    for k in range(args.steps):
        dt, c = pool.run(inputs_base_seed() + 3 + k * workers)
        times.append(dt)
        cpu += c
    pool.close()
    ms = 1e3 * statistics.mean(times)
    value = workers / (ms * 1e-3)
    cores = cores_used(sum(times), cpu)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": ws,
        "devices": "host cores only: the oracle runs on rank 0's CPU and uses no GPU",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"SGL inverse+forward, B={B_BENCH}, batch {BATCH} functions per GPU",
                   "B": B_BENCH, "batch": BATCH, "precision": "fp64 (oracle)",
                   "step_sample": f"{workers} functions of the batch per step, one per worker process"},
        "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": cores, "kind": "oracle",
                         "threads_available": os.cpu_count(), "cpu_s": cpu,
                         "sample": f"{workers} whole functions of B=128 per step (inverse + forward), "
                                   f"{workers} processes of one BLAS thread, FP64 NumPy"},
        "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def inputs_base_seed():
    from paper_1604_05140_gb300 import inputs
    return inputs.BASE_SEED


def relaunch(args):
    """`--gpus N` with N > 1 outside a launcher: run this script again as N
    ranks under torch.distributed.run (one process per GPU, rendezvous on
    127.0.0.1) and return its exit status; None when no relaunch is needed."""
    if args.gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def error_gate(line):
    """Names of the round-trip error bounds the line misses: 1e-12 normwise
    for the FP64 path, 1e-6 for the split-precision (tensor-core, three
    product) paths; empty when every bound holds."""
    bounds = {"fp64": 1e-12, "tf32x3": 1e-6, "fp16x3": 1e-6}
    missed = []
    prec = line["config"]["precision"]
    if prec in bounds and line["round_trip_errors"]["normwise_max"] > bounds[prec]:
        missed.append(f"{prec} round trip {line['round_trip_errors']['normwise_max']:.3g} > {bounds[prec]:g}")
    fp = line.get("fp64_path")
    if fp and fp["round_trip_errors"]["normwise_max"] > bounds["fp64"]:
        missed.append(f"fp64 round trip {fp['round_trip_errors']['normwise_max']:.3g} > 1e-12")
    for name, v in line.get("variants", {}).items():
        e = v["round_trip_errors"]["normwise_max"] if "round_trip_errors" in v else v["round_trip_max_rel_err"]
        if name in bounds and e > bounds[name]:
            missed.append(f"{name} round trip {e:.3g} > {bounds[name]:g}")
    return missed


def main():
    global BATCH, TUNE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["tf32x3", "tf32", "bf16x3", "fp16x3", "fp32", "fp64"])
    ap.add_argument("--no-variants", action="store_true", help="skip the reduced-precision variant lines")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=16.0,
                    help="CPU baseline budget, split between one core and all cores")
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="oracle worker processes of the all-cores baseline and the reference arm (0: one per core)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--profile-case", choices=["uneven", "uniform", "paper_grid", "midpoint"], default=None,
                    help="run only this workload's round trips (for profiler captures) and exit")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="functions per GPU (64 is the benchmark workload; smaller only for profiling runs)")
    args = ap.parse_args()
    BATCH = args.batch
    TUNE = not args.no_autotune
    if args.profile_case:
        profile_case(args.profile_case, args.precision, args.steps, args.warmup)
        return
    rc = relaunch(args)
    if rc is not None:
        sys.exit(rc)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
