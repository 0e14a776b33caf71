"""The benchmark's multi-GPU path is replicas only: under torchrun every rank
fixes its own configuration (seed + rank) with no collective on the data
path.  What crosses ranks is the timing: a barrier around each timed region,
the maximum of the ranks' times, and a value counting the units of all
ranks.  These tests run that host logic as two gloo ranks on the CPU."""
import argparse
import json
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch

    import bench
    rp = bench.Replicas("gloo", torch.device("cpu"))
    rp.barrier()
    mine = 1.0 + 0.5 * rank  # the last rank is the slowest
    slowest = rp.max(mine)
    res = {"rank": rank, "world": rp.world, "max": slowest, "seed": rp.seed(7),
           "value": rp.throughput(1000.0, slowest)}
    rp.barrier()
    rp.close()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_time_the_slowest_rank_and_count_all_units(tmp_path, world):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{k}.json")) for k in range(world)]
    slowest = 1.0 + 0.5 * (world - 1)
    for k, r in enumerate(res):
        assert r["world"] == world
        assert r["max"] == slowest
        assert r["seed"] == 7 + k  # independent configurations
        assert r["value"] == pytest.approx(world * 1000.0 / slowest)


def test_single_process_needs_no_process_group(monkeypatch):
    import torch

    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rp = bench.Replicas("gloo", torch.device("cpu"))
    assert (rp.world, rp.rank) == (1, 0)
    assert rp.max(2.5) == 2.5 and rp.seed(3) == 3 and rp.throughput(10.0, 2.0) == 5.0
    rp.barrier()
    rp.close()


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    """Under torchrun the oracle arm runs and prints on rank 0; the other ranks
    return at once without work."""
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, bench.WORKLOADS[bench.DEFAULT_WORKLOAD]) is None


def test_reference_arm_line_on_rank_0(monkeypatch):
    """On rank 0 the oracle arm prints one JSON line with the same metric and
    config as the GPU arm, a cpu_baseline describing its sample and an e2e
    equal to its value (the oracle's cost is stubbed: this checks the line,
    not the oracle's speed)."""
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "time_oracle", lambda U, n, alpha, threads=1: 1e-6 * max(n, 1) * U.shape[0])
    monkeypatch.setattr(bench, "host_cores", lambda: 4)
    args = argparse.Namespace(steps=2, warmup=1)
    W = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    line = bench.run_reference(args, W)
    assert line is not None
    json.dumps(line)  # serialisable
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["config"] == bench.main_config(W, 1, W["dtype"].startswith("f32"))
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 4
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["steps"] == 2 and line["warmup"] == 1
