"""Sharding a sweep or batch of independent domains over the ranks of a job.

Domains are independent until their permeabilities are collected, so a job
with several GPUs splits the domain list: each rank solves its share as one
batch on its own GPU, and the only collective is gathering the k values at
the end.  The split is longest-processing-time first (Graham 1969): domains
sorted by estimated cost, each given to the least-loaded rank; the largest
load is at most 4/3 of the optimum.

The cost estimate is the fluid-node updates to steady state, taken as
cells x N_x x (1 + 2 (tau - 1/2)): the pressure field relaxes over a time
that grows with the domain length, and the measured steps to steady state
grow with tau (a heuristic only; the split is correct for any cost).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Optional, Sequence

import numpy as np


def domain_cost(shape: Sequence[int], tau: float) -> float:
    """Estimated work of one domain (see the module docstring)."""
    nx = int(shape[-1])
    cells = int(np.prod(shape))
    return float(cells) * nx * (1.0 + 2.0 * (tau - 0.5))


def lpt_partition(costs: Sequence[float], nparts: int) -> List[List[int]]:
    """Indices of `costs` split into `nparts` lists, longest-processing-time
    first; each list keeps ascending index order."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, p) for p in range(nparts)]
    parts: List[List[int]] = [[] for _ in range(nparts)]
    for i in order:
        load, p = heapq.heappop(heap)
        parts[p].append(i)
        heapq.heappush(heap, (load + float(costs[i]), p))
    return [sorted(p) for p in parts]


def _solve_on_gpu(masks, taus, drhos, tol, max_steps):
    from . import lbm
    if not masks:
        return np.zeros(0), np.zeros(0, np.int32)
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        _, st, _, _ = lbm.lbm_run_to_steady(s, tol, max_steps)
        k, _ = lbm.lbm_permeability(s)
    return np.asarray(k, np.float64), np.asarray(st, np.int32)


def solve_sharded(masks: Sequence[np.ndarray], taus: Sequence[float], drhos: Sequence[float],
                  tol: float = 1e-9, max_steps: int = 2_000_000, group=None,
                  solve: Optional[Callable] = None):
    """Solve every domain to steady state, sharded over the ranks of the
    default (or given) torch.distributed process group; every rank returns
    (k, status) for all domains in the input order.  Without an initialised
    process group the whole list runs on this process.  `solve(masks, taus,
    drhos, tol, max_steps) -> (k, status)` replaces the GPU solver (tests)."""
    solve = solve or _solve_on_gpu
    n = len(masks)
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return solve(list(masks), list(taus), list(drhos), tol, max_steps)
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    parts = lpt_partition([domain_cost(m.shape, t) for m, t in zip(masks, taus)], world)
    mine = parts[rank]
    k, st = solve([masks[i] for i in mine], [taus[i] for i in mine], [drhos[i] for i in mine], tol, max_steps)
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, [float(v) for v in k], [int(v) for v in st]), group=group)
    k_all = np.full(n, np.nan)
    st_all = np.zeros(n, np.int32)
    for idx, kk, ss in gathered:
        k_all[idx] = kk
        st_all[idx] = ss
    return k_all, st_all
