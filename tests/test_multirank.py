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


def _sweep_reports(indices, n_samples):
    """One controller step of each listed sample of a small FOM-FOM sweep, advanced by the oracle (the
    per-instance work of the sharded batched sweep, on the CPU): {sample: (status, iterations, |u|)}."""
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import oracle as O
    from paper_2511_20687_gb300 import workloads as W
    specs = W.batched_samples(n_samples=n_samples, n_min=2, n_max=3, rom=False)
    out = {}
    for i in indices:
        sp = specs[i]
        sp.n_substeps = 4
        prob = O.Problem(sp)
        r = prob.step()
        out[i] = (r["status"], r["iterations"], float(np.linalg.norm(prob.state(1)[0])))
    return out


def _sweep_rank_main(rank, world, port, n_samples, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2511_20687_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = W.batched_samples(n_samples=n_samples, n_min=2, n_max=3, rom=False)
        mine = bench.shard_samples([sp.subdomains[0].n_elements for sp in specs], world)[rank]
        out[rank] = (mine, bench.gather_reports(_sweep_reports(mine, n_samples)))
    finally:
        dist.destroy_process_group()


def test_shard_samples_covers_every_sample_once_and_balances_elements():
    sys.path.insert(0, ROOT)
    import bench
    sizes = [((7 * i) % 25 + 8) ** 3 for i in range(256)]
    for world in (1, 2, 3, 8):
        parts = bench.shard_samples(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)


def test_sharded_sweep_gloo_world_size_2_equals_single_process():
    """Each rank advances only its shard and the gathered per-instance reports equal those of one
    process advancing every sample (no data-path exchange: the gather is the only collective)."""
    n = 6
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_sweep_rank_main, args=(2, _free_port(), n, out), nprocs=2, join=True,
                           start_method="spawn")
        got = dict(out)
    single = _sweep_reports(range(n), n)
    assert sorted(got[0][0] + got[1][0]) == list(range(n)) and not set(got[0][0]) & set(got[1][0])
    assert got[0][1] == single and got[1][1] == single
