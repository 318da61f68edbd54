"""The benchmark's multi-process path on CPU: with N ranks every rank runs its own
replica, the job time is the slowest rank's and the work is the sum over ranks
(gloo backend, world size 2, no GPU)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, units = bench.reduce_over_ranks(10.0 * (rank + 1), 1000.0 * (rank + 1))
    out.put((rank, ms, units))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == 20.0 and units == 3000.0


def test_single_process_is_unchanged():
    import bench

    assert bench.reduce_over_ranks(5.0, 7.0) == (5.0, 7.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus, workload = 3, 1, 2, "channel_1m"

    assert bench.run_reference(A()) == 0
