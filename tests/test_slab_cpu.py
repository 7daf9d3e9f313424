"""One domain cut into x-slabs with a halo exchange after every step, on the
CPU: the FP64 oracle steps each slab on its columns plus ghost columns, and the
library's slab driver (paper_1609_09685_gb300/slabs.py) exchanges the cuts --
inside one process, and between gloo ranks.  The sliced run must equal the
whole-domain oracle bit for bit, and the permeability from the summed link
flux must equal the whole domain's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from oracle.slab import OracleSlab
from paper_1609_09685_gb300 import slabs


def test_split_and_extent():
    assert slabs.split_columns(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slabs.split_columns(5, 1) == [(0, 5)]
    with pytest.raises(ValueError):
        slabs.split_columns(3, 4)
    assert slabs.slab_extent(0, 4, 10) == (0, 5, 2)
    assert slabs.slab_extent(4, 7, 10) == (3, 5, 3)
    assert slabs.slab_extent(7, 10, 10) == (6, 4, 1)
    assert slabs.slab_extent(0, 10, 10) == (0, 10, 0)
    m = np.arange(2 * 3 * 10).reshape(2, 3, 10).astype(np.uint8) % 2
    assert np.array_equal(slabs.slab_mask(m, 4, 7), m[..., 3:8])


def _case(dim):
    rng = np.random.default_rng(50 + dim)
    if dim == 2:
        mask = (rng.random((9, 23)) < 0.3).astype(np.uint8)
    else:
        mask = (rng.random((4, 5, 17)) < 0.3).astype(np.uint8)
    return mask, 0.8, 1e-3


def _assemble(parts, mask):
    return np.concatenate(parts, axis=mask.ndim - 1)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("parts", [2, 3])
def test_slabs_in_one_process_equal_the_whole_domain(dim, parts):
    mask, tau, drho = _case(dim)
    nx = mask.shape[-1]
    sl = [OracleSlab(mask, lo, hi, tau, drho) for lo, hi in slabs.split_columns(nx, parts)]
    drv = slabs.SlabDriver(sl, 0, parts)
    drv.step(12)
    whole = O.run(mask, O.init(mask, 1 + drho, 1.0), tau, 1 + drho, 1.0, 12)
    assert np.array_equal(_assemble([s.real() for s in sl], mask), whole)
    k, _, _ = drv.observe()
    assert k == pytest.approx(O.permeability(mask, whole, tau, 1 + drho, 1.0), rel=1e-13)


def test_a_missing_exchange_is_detected():
    """The check has teeth: without the exchange the slabs drift apart from
    the whole domain."""
    mask, tau, drho = _case(2)
    sl = [OracleSlab(mask, lo, hi, tau, drho) for lo, hi in slabs.split_columns(mask.shape[-1], 2)]
    for _ in range(6):
        for s in sl:
            s.step(1)
    whole = O.run(mask, O.init(mask, 1 + drho, 1.0), tau, 1 + drho, 1.0, 6)
    assert not np.array_equal(_assemble([s.real() for s in sl], mask), whole)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, dim, nslab, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mask, tau, drho = _case(dim)
        cols = slabs.split_columns(mask.shape[-1], nslab)
        owner = [min(j * world // nslab, world - 1) for j in range(nslab)]
        mine = [j for j in range(nslab) if owner[j] == rank]
        sl = [OracleSlab(mask, *cols[j], tau, drho) for j in mine]
        drv = slabs.SlabDriver(sl, mine[0], nslab, owner=owner, dist=dist)
        drv.step(10)
        k, _, _ = drv.observe()
        q.put((rank, mine, [s.real() for s in sl], k))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nslab,dim", [(2, 2, 2), (3, 3, 2), (2, 4, 3)])
def test_slabs_on_gloo_ranks_equal_the_whole_domain(world, nslab, dim):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, dim, nslab, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mask, tau, drho = _case(dim)
    parts = [r for (_, _, reals, _) in out for r in reals]
    whole = O.run(mask, O.init(mask, 1 + drho, 1.0), tau, 1 + drho, 1.0, 10)
    assert np.array_equal(_assemble(parts, mask), whole)
    k_whole = O.permeability(mask, whole, tau, 1 + drho, 1.0)
    for (_, _, _, k) in out:
        assert k == pytest.approx(k_whole, rel=1e-13)
