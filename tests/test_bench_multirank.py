"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would
start them. Each rank runs its own replica (its own shot), the elapsed time is
the maximum over ranks, and the whole-job value counts every rank's nodes."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        workload, n = "graded", 16
    m = bench.workload(A(), rank)
    el = 1.0 + 0.5 * rank                       # the slower rank sets the job time
    el_max = bench.max_over_ranks(torch, dist, el, world, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, tuple(m["src_xy"]))
    if rank == 0:
        out.put((el_max, bench.job_rate(world, 1000, 10, el_max), gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_replicas():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    el_max, rate, srcs = out.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert el_max == 1.5
    assert rate == pytest.approx(2 * 1000 * 10 / 1.5)
    assert srcs[0] != srcs[1]                    # each rank shoots from its own source


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, dist, 2.5, 1, "cpu") == 2.5
