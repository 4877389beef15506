"""The multi-process path of bench.py on CPU: two gloo ranks, each timing its
own replica, agree on the slowest rank's time (the job is as slow as its
slowest GPU); the reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [3.5, 7.25][rank]
        q.put((rank, bench.max_over_ranks(mine, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 7.25, 1: 7.25}


def test_single_rank_is_identity():
    assert bench.max_over_ranks(2.5, 1) == 2.5


def test_reference_arm_only_rank0_works(capsys):
    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A, 2, 1)  # rank 1: returns at once, prints nothing
    assert capsys.readouterr().out == ""
