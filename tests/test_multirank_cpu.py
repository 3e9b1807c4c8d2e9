"""The multi-GPU path of bench.py is replicas only: every rank propagates its
own evidence cases, the ranks meet only to take the slowest rank's time, and
the job's rate counts every rank's cases.  Checked with two gloo processes on
the CPU (no GPU, no NCCL)."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.job_rate(1000, 64, world, ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate, "seed": bench.evidence_seed(rank)}, f)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.loads((tmp_path / f"r{i}.json").read_text()) for i in range(world)]
    # every rank sees the slowest rank's time, and the job's rate counts both
    # ranks' cases over it
    assert r[0]["ms"] == r[1]["ms"] == 15.0
    assert r[0]["rate"] == pytest.approx(1000 * 64 * world / 15e-3)
    assert r[0]["rate"] == r[1]["rate"]
    # each replica propagates its own evidence cases
    assert r[0]["seed"] != r[1]["seed"]


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(10, 4, 1, 2.0) == pytest.approx(10 * 4 / 2e-3)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under torchrun the FP64 oracle arm runs on rank 0 alone; the other
    ranks exit at once without output."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, batch=64, no_serving=True, impl="reference",
                              no_cpu_baseline=True)
    assert bench.run_reference(args, 1, 2) == 0
    assert capsys.readouterr().out == ""
