"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): each rank
gets its own independent domains and the whole-job figures take the slowest
rank's time and the sum of the ranks' work.  No data-path collective exists."""
import os
import socket

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
