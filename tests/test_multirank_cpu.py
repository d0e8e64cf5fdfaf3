"""Host logic of the multi-rank benchmark path on CPU with two gloo ranks:
each rank takes its own seeded system, the step time is the maximum over
ranks and the throughput counts the particles of every rank."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        w = bench.rank_workload(bench.WORKLOAD, rank)
        ms, n_all = bench.reduce_timing(dist, 10.0 + rank, w["n"] // (rank + 1))
        out[rank] = (w["seed"], ms, n_all)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_systems_and_take_the_slowest():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    import bench

    n = bench.WORKLOAD["n"]
    assert out[0][0] != out[1][0]                 # different systems per rank
    assert out[0][1] == out[1][1] == 11.0         # max over ranks
    assert out[0][2] == out[1][2] == n + n // 2   # particles of all ranks
