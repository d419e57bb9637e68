"""The bench's multi-rank path on the CPU: world_size-2 gloo process groups over
127.0.0.1.  A weakly scaled job's time is its slowest rank's, and its rate counts every
rank's units; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 10.0 + 5.0 * rank                  # rank 1 is the slower one
    slowest = bench.max_over_ranks(local, world, device="cpu")
    q.put((rank, slowest, bench.job_rate(1000, 3, world, slowest / 1000.0)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in out:
        assert slowest == 15.0                  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000 * 3 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.job_rate(10, 2, 1, 0.5) == 40.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="cfg0", mode="hogwild", steps=1, warmup=0, cpu_sample=100)
    bench.run_reference(args, world=2, rank=1)          # returns at once, prints nothing
    assert capsys.readouterr().out == ""
