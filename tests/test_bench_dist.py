"""Host logic of the multi-process benchmark (one process per GPU, replicas
of the workload): the rank environment, and the whole-job step time taken as
the maximum over ranks, on two gloo processes on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w, r, lr = bench.dist_env()
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    out[rank] = (w, r, lr, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_step():
    import torch.multiprocessing as mp

    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank, (w, r, lr, slowest) in res.items():
        assert (w, r, lr) == (world, rank, rank)
        assert slowest == 15.0


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
