"""The multi-GPU form of the benchmark is replicas only: each rank builds its
own cloud and the ranks exchange nothing but the step time.  Two gloo ranks on
the CPU check that the job's step time is the slowest rank's and the rate
counts every rank's points, and that a rank leaving before the collective
makes the other's collective fail instead of hang."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, ms_of_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, rate = bench.replica_rate(ms_of_rank[rank], 1_000_000, world, torch.device("cpu"))
        out.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    ms_of_rank = [10.0, 12.5]
    procs = [ctx.Process(target=worker, args=(r, 2, port, ms_of_rank, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 12.5                                      # the slowest rank decides
        assert rate == pytest.approx(2 * 1_000_000 / 12.5e-3 / 1e9)   # both ranks' points


def leaving_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:   # leaves between steps, before the collective
        dist.destroy_process_group()
        out.put((rank, "left"))
        return
    try:
        bench.replica_rate(10.0, 1000, world, torch.device("cpu"))
        out.put((rank, "completed"))
    except Exception as ex:   # the collective ends with an error instead of waiting forever
        out.put((rank, "error: " + type(ex).__name__))


def test_rank_leaving_fails_the_collective():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=leaving_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "left"
    assert res[0].startswith("error"), res[0]
