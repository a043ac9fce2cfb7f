"""Host logic of bench.py across ranks, on the CPU with gloo (world size 2):
each rank solves its own system (seeds differ), the slowest rank's time and
the iterations of all ranks make the whole-job figure, and the reference arm
prints only on rank 0."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total_s = 1.0 + rank          # rank 1 is the slower one
        iters = 100 * (rank + 1)
        t, it = bench.aggregate(total_s, iters, dist, "cpu")
        r, w, _ = bench.dist_env()
        out[rank] = (t, it, r, w)
    finally:
        dist.destroy_process_group()


def test_aggregate_takes_slowest_time_and_all_iterations():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, it, r, w = res[rank]
        assert (r, w) == (rank, world)
        assert t == 2.0 and it == 300.0


def test_aggregate_single_process():
    assert bench.aggregate(1.5, 7) == (1.5, 7.0)


def test_ranks_get_distinct_systems():
    a = bench.make_system_small(0)
    b = bench.make_system_small(1)
    assert a.b.shape == b.b.shape and not (a.b == b.b).all()


def test_reference_arm_prints_only_on_rank0(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
