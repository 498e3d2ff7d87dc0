"""Multi-process path of bench.py on the host: replicas over gloo.

The transform of one function never needs another function's data, so
several GPUs run independent replicas; the only exchange is the max of the
ranks' step times for the whole-job number.  Two gloo ranks on the CPU check
that reduction, the aggregation, and that the reference arm runs on rank 0
only.
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
        steps, warmup = 1, 0

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    # rank 0 times one whole B=128 function through the oracle and prints one
    # JSON line with the contract's keys (a few seconds of CPU work)
    sys.path.insert(0, ROOT)
    import json
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 1

    monkeypatch.setenv("RANK", "0")
    bench.run_reference(Args())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    # cores: the threads the oracle kept busy (CPU time over wall time), not the pool size
    cb = line["cpu_baseline"]
    assert 1 <= cb["cores"] <= cb["threads_available"] and cb["cpu_s"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
