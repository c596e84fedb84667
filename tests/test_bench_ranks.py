"""Host logic of bench.py's multi-process form, on CPU: replicas under a gloo process group
(world size 2) agree on the slowest rank's time, and the whole-job value counts every rank's
node updates; the reference arm does its work on rank 0 only."""
import argparse
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        job_ms = bench.max_over_ranks(local_ms, "cpu")
        value = bench.whole_job_mlups(1024 * 1024, 20, world, job_ms)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"local_ms": local_ms, "job_ms": job_ms, "value": value}, fh)
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [r["job_ms"] for r in res] == [15.0, 15.0]
    assert res[0]["value"] == res[1]["value"] == pytest.approx(2 * 1024 * 1024 * 20 / 15e-3 / 1e6)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.whole_job_mlups(100, 10, 1, 1.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=2, warmup=1, gpus=2, impl="reference")
    assert bench.reference_main(args) == 0
    assert capsys.readouterr().out == ""
