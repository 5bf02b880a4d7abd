"""The multi-rank path of bench.py on CPU: two gloo ranks (one process each, as torchrun starts
them) reduce their timed-region lengths to the slowest rank's, and the whole-job throughput counts
every rank's replica (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 25.0 * rank  # rank 1 is the slowest
    got = bench.max_over_ranks(ms, world, torch.device("cpu"))
    out[rank] = (got, bench.job_throughput(1000, 4, world, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_replica():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        got, thr = res[rank]
        assert got == 125.0
        assert thr == pytest.approx(world * 1000 * 4 / 0.125)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, 1, None) == 7.5
    assert bench.job_throughput(10, 2, 1, 1000.0) == 20.0
