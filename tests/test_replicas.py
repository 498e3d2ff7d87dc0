"""Multi-process path of bench.py on the host: replicas over gloo.

The transform of one function never needs another function's data, so
several GPUs run independent replicas; the only exchange is the max of the
ranks' step times for the whole-job number.  Two gloo ranks on the CPU check
that reduction, the aggregation, and that the reference arm runs on rank 0
only; `bench.py --gpus 2` run as one command starts both ranks itself.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import bench
    got_ws, got_rank, _ = bench.dist_setup()
    import torch.distributed as dist
    assert dist.get_backend() == "gloo"
    bench.barrier(got_ws)
    # rank r pretends its step took 10 + 5 r ms for 64 functions
    value, ms = bench.whole_job(got_ws, 64, 10.0 + 5.0 * rank)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{got_ws} {got_rank} {value!r} {ms!r}\n")
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_gloo_ranks_whole_job(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(ws)]
    slowest = 10.0 + 5.0 * (ws - 1)
    for r, (gws, grank, value, ms) in enumerate(rows):
        assert int(gws) == ws and int(grank) == r
        assert float(ms) == slowest                       # every rank sees the slowest rank's time
        assert float(value) == pytest.approx(ws * 64 / (slowest * 1e-3))  # all functions / that time


def test_single_process_is_identity(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.whole_job(1, 64, 8.0) == (pytest.approx(8000.0), 8.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, cpu_workers = 1, 0, 1

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def _bench(*argv, timeout=300):
    import subprocess
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], capture_output=True, text=True,
                          timeout=timeout, env=env, cwd=ROOT)


@pytest.mark.timeout(400)
def test_reference_arm_with_two_ranks_from_one_command():
    # `bench.py --gpus 2` outside a launcher starts two ranks itself (torch
    # distributed run); rank 0 alone times the oracle (one whole B=128
    # function per step here) and prints one line that counts both ranks
    import json
    sys.path.insert(0, ROOT)
    import bench
    r = _bench("--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-workers", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["n_gpus"] == 2
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"]
    assert 1 <= cb["cores"] <= cb["threads_available"] and cb["cpu_s"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


@pytest.mark.timeout(200)
def test_gpu_arm_refuses_more_ranks_than_gpus():
    # two ranks on a host without GPUs: every rank stops with a message and a
    # non-zero status instead of running replicas on the wrong device
    r = _bench("--gpus", "2", "--steps", "1", "--warmup", "3", "--no-cpu")
    assert r.returncode != 0
    assert "need as many visible GPUs" in r.stderr


def test_cpu_baseline_one_and_all_cores():
    # the oracle on one core and in two worker processes (small bandlimit to
    # keep the test short); both figures are reported
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_oracle_sample(B=8, budget_s=0.4, workers=2)
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] > 0
    assert cb["one_thread"]["cores"] == 1 and cb["one_thread"]["value"] > 0
    assert "2 processes" in cb["sample"]
