"""The benchmark's multi-rank path on CPU: two gloo ranks aggregate their
timings as the GPU run does (units summed over ranks, slowest rank's time),
and the reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r processed 1000 (r + 1) units in 10 (r + 1) ms
    value, max_ms = bench.job_throughput(1000.0 * (rank + 1), 10.0 * (rank + 1), world, device="cpu")
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"value": value, "max_ms": max_ms}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_gpu_run(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got["max_ms"] == 20.0
        assert got["value"] == pytest.approx((1000.0 + 2000.0) / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(500.0, 10.0, 1) == (50000.0, 10.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})())
    assert capsys.readouterr().out == ""
