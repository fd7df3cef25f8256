"""The N > 1 bookkeeping of bench.py (replicas: max of the timed milliseconds, sum of the element-
updates and of the kernel launches over ranks) on two CPU ranks with the gloo backend."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pairs = [(10.0 + rank, 1000 * (rank + 1)), (5.0 * (2 - rank), 7)]
        launches = bench.combine_ranks([(0.0, 1107 + rank)], "cpu")   # the gpu_launches reduction
        out[rank] = (bench.combine_ranks(pairs, "cpu"), launches)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        got = dict(out)
    expect = ([(11.0, 3000), (10.0, 14)], [(0.0, 2215)])
    assert got[0] == expect and got[1] == expect


def test_combine_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks([(3.5, 12)], "cpu") == [(3.5, 12)]
