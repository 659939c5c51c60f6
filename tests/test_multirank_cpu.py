"""The benchmark's multi-rank host logic on CPU, world size 2 over gloo: each rank draws its own
seeded batch of the same family (weak scaling, no data-path collective), and the whole-job
figures are the slowest rank's time and the sum of the units all ranks processed."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1602_00182_gb300 import inputs as I
        inst = I.burgers_batch(count=16, seed_index=bench.rank_seed(1, rank))
        sig = torch.tensor([float(sum(it.n for it in inst)), float(inst[0].u0.sum())], dtype=torch.float64)
        sigs = [torch.zeros_like(sig) for _ in range(world)]
        dist.all_gather(sigs, sig)
        t, u = bench.job_totals(10.0 * (rank + 1), 1000 * (rank + 1), world, torch.device("cpu"))
        q.put((rank, [s.tolist() for s in sigs], t, u, [it.n for it in inst]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every rank sees the same gathered signatures, and the two batches differ
    assert res[0][1] == res[1][1]
    assert res[0][1][0] != res[0][1][1]
    # max time over ranks, sum of units over ranks, identical on both ranks
    for _, _, t, u, _ in res:
        assert t == 20.0 and u == 3000.0
    # both batches are drawn from the same family (N within the configured range)
    for _, _, _, _, ns in res:
        assert min(ns) >= 64 and max(ns) <= 8192


def test_single_rank_totals_are_local():
    import bench
    assert bench.job_totals(12.5, 77, 1, None) == (12.5, 77)
    assert bench.rank_seed(1, 0) == 1 and bench.rank_seed(1, 3) != bench.rank_seed(2, 3)
