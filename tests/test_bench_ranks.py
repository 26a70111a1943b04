"""Host logic of bench.py's N-rank runs (one process per GPU, each solving its
own replica of the workload): the job's time is the slowest rank's, the
job's throughput adds up the replicas, and the reference arm (the oracle on
the host cores) runs on rank 0 only.  The multi-rank parts run as two gloo
processes on the CPU."""
import json
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    t = b.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
    v = b.job_gdofs(world, 100663296, 7, t)
    dist.barrier()
    dist.destroy_process_group()
    with open(f"{out}.{rank}", "w") as f:
        json.dump({"t": t, "v": v}, f)


def test_two_ranks_take_the_slowest_time_and_add_the_replicas(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "rank")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(f"{out}.{r}"))
        assert d["t"] == 1.5
        assert abs(d["v"] - 2 * 100663296 * 7 / 1.5 / 1e9) < 1e-12


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.25, None) == 0.25
    assert bench.job_gdofs(1, 1e9, 3, 1.5) == 2.0


def _fake_baseline(calls):
    def baseline():
        calls.append(1)
        return {"value": 1.0e-4, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
                "sample": "fake"}
    return baseline


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    args = types.SimpleNamespace(warmup=3, steps=2, gpus=2)
    calls = []
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(args, baseline=_fake_baseline(calls)) == 0
    assert calls == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    assert bench.run_reference(args, baseline=_fake_baseline(calls)) == 0
    assert len(calls) == 5  # three untimed warm-up samples, two timed
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["value"] == 1.0e-4
    assert line["e2e"] == {"value": 1.0e-4, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["ms_per_step"] >= 0.0
