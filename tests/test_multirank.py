"""Replica sharding across ranks (world size 2, gloo, CPU): disjoint primary ranges
merged on rank 0 equal one run over the union."""
import os
import socket

import numpy as np
import pytest

from paper_1806_00205_gb300 import shard


def test_merge_results_adds_exactly():
    a = {k: 3 for k in shard.INT_KEYS}
    b = {k: 5 for k in shard.INT_KEYS}
    a.update(e_sum=1.5, e2_sum=2.5, hist_e=[1, 2], hist_a=[0, 1], hist_z=[7, 0, 1])
    b.update(e_sum=0.5, e2_sum=0.5, hist_e=[3, 4], hist_a=[2, 2], hist_z=[1, 1, 1])
    m = shard.merge_results([a, b])
    assert m["rays"] == 8 and m["sum_k"] == 8 and m["e_sum"] == 2.0 and m["hist_e"] == [4, 6]
    assert m["hist_z"] == [8, 1, 2]
    assert m["sey"] == 1.0
    assert shard.primary_offset(3, 1000, 7) == 3007


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1806_00205_gb300 import inputs as I
    mesh = I.grf_foam(12, 0.5, 2.0, seed=21)
    r = O.run(mesh, I.see_table(), 400.0, 30.0, n, seed=99, primary_offset=shard.primary_offset(rank, n),
              n_threads=1)
    merged = shard.gather_merge(r)
    if rank == 0:
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_run():
    import torch.multiprocessing as mp
    import oracle as O
    from paper_1806_00205_gb300 import inputs as I
    n = 400
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mesh = I.grf_foam(12, 0.5, 2.0, seed=21)
    full = O.run(mesh, I.see_table(), 400.0, 30.0, 2 * n, seed=99, n_threads=1)
    for k in shard.INT_KEYS:
        assert merged[k] == full[k], k
    assert merged["hist_e"] == full["hist_e"].tolist()
    assert abs(merged["e_sum"] - full["e_sum"]) <= 1e-9 * max(1.0, full["e_sum"])
    assert merged["sey"] == full["sey"]


def _timing_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 10 + 5 r ms and traced 1000 (r + 1) rays of 100 primaries
    ms, counts = shard.reduce_timing(10.0 + 5.0 * rank, [1000.0 * (rank + 1), 100.0], device="cpu")
    q.put((rank, ms, counts))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_timing_takes_the_slowest_rank_and_sums_the_work():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_timing_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, counts in got:                 # every rank sees the whole-job numbers
        assert ms == 15.0 and counts == [3000.0, 200.0]
    # throughput as the bench reports it: summed work over the slowest rank's time
    assert counts[0] / (ms / 1e3) == 200000.0


def test_reduce_timing_without_a_process_group_is_the_identity():
    assert shard.reduce_timing(12.5, [7, 3]) == (12.5, [7.0, 3.0])
