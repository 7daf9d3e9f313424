"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): each rank
gets its own independent domains and the whole-job figures take the slowest
rank's time and the sum of the ranks' work.  No data-path collective exists."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = bench.get_workload("sweep", rank)
    seeds = sorted({d.seed for d in wl.domains})
    t = 1.0 + rank            # this rank's time
    work = 100.0 * (rank + 1)  # this rank's updates
    mx, sm = bench.combine_ranks(dist, "cpu", [t, 0.5 * t], [work])
    q.put((rank, seeds, mx, sm, len(wl.domains)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_combination():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, mx0, sm0, n0), (r1, s1, mx1, sm1, n1) = out
    assert s0 != s1                      # independent domains per rank
    assert n0 == n1 == 24                # same amount of work per rank (weak scaling)
    assert mx0 == mx1 == [2.0, 1.0]      # slowest rank's time
    assert sm0 == sm1 == [300.0]         # total work of the job


# --------------------------------------------------------------------------
# Sharding a sweep over ranks (paper_1609_09685_gb300/sharding.py)
# --------------------------------------------------------------------------

def test_lpt_partition_covers_every_domain_once_within_the_graham_bound():
    import itertools

    from paper_1609_09685_gb300 import sharding
    rng = np.random.default_rng(3)
    for trial in range(20):
        costs = list(rng.integers(1, 50, size=9).astype(float))
        for parts_n in (1, 2, 3):
            parts = sharding.lpt_partition(costs, parts_n)
            assert sorted(i for p in parts for i in p) == list(range(9))
            loads = [sum(costs[i] for i in p) for p in parts]
            # brute-force optimum of the largest load
            best = min(max(sum(c for c, a in zip(costs, assign) if a == b) for b in range(parts_n))
                       for assign in itertools.product(range(parts_n), repeat=9)) if parts_n > 1 else sum(costs)
            assert max(loads) <= 4.0 / 3.0 * best + 1e-9


def _fake_solve(masks, taus, drhos, tol, max_steps):
    # a stand-in for the GPU solver: k from the domain's shape and tau
    k = np.array([m.shape[-1] + 1000.0 * t for m, t in zip(masks, taus)])
    return k, np.zeros(len(masks), np.int32)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1609_09685_gb300 import sharding
    shapes = [(20, 40), (50, 100), (10, 30), (60, 120), (30, 60)]
    masks = [np.zeros(s, np.uint8) for s in shapes]
    taus = [0.6, 0.9, 1.2, 0.7, 1.5]
    k, st = sharding.solve_sharded(masks, taus, [1e-3] * 5, solve=_fake_solve)
    q.put((rank, [float(v) for v in k], [int(v) for v in st]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_sweep_gathers_every_k_in_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = [40 + 600.0, 100 + 900.0, 30 + 1200.0, 120 + 700.0, 60 + 1500.0]
    for rank, k, st in out:
        assert k == expect and st == [0] * 5
