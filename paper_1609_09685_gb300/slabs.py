"""One domain cut into x-slabs, one solver per slab, with a halo exchange
after every step (the domain decomposition of the method of Sec. 2 for a
domain larger than one GPU).

The slabs of a domain are numbered left to right; a process (rank of
`torch.distributed`, or the only process) holds a consecutive run of them.
After every step each cut between slab j and j + 1 is exchanged: slab j packs
its last real column's c_x = +1 planes for slab j + 1's left ghost column,
slab j + 1 its first real column's c_x = -1 planes for slab j's right ghost
(lbm_slab_export / lbm_slab_import).  A cut inside a process is a copy through
a device buffer; a cut between processes is a point-to-point send and receive
of that buffer (NCCL for GPU buffers, gloo for host buffers).  Observables are
summed over the slabs (slot 3 is a maximum) -- the only collective -- and the
solver turns the sums into the whole domain's permeability, Kn and residual
(lbm_slab_observables).  No method arithmetic happens here: the steps, the
packing and the Darcy law run in the library's kernels and C code.

The driver is written against a small slab interface (step,
halo_floats(side, incoming), export, import_, observe, finalize, new_buffer),
implemented here by `GpuSlab` on the library; the CPU tests drive the FP64
oracle through the same interface on gloo ranks.  GPU slabs run on torch's
current stream by default, so that the exports, the buffer copies or
transfers and the imports are ordered without host synchronisation.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def split_columns(nx: int, parts: int) -> List[Tuple[int, int]]:
    """Real column ranges [lo, hi) of `parts` slabs, as even as possible."""
    if parts < 1 or parts > nx:
        raise ValueError("need 1 <= parts <= nx")
    base, extra = divmod(nx, parts)
    out, lo = [], 0
    for j in range(parts):
        hi = lo + base + (1 if j < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def slab_extent(lo: int, hi: int, nx: int) -> Tuple[int, int, int]:
    """(x_offset, columns including ghosts, ghost bits) of real columns [lo, hi)."""
    left = 1 if lo > 0 else 0
    right = 1 if hi < nx else 0
    return lo - left, hi - lo + left + right, left | (right << 1)


def slab_mask(mask: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """The whole mask's columns of a slab, ghosts included (x is the last axis)."""
    x0, n, _ = slab_extent(lo, hi, mask.shape[-1])
    return np.ascontiguousarray(mask[..., x0:x0 + n])


class GpuSlab:
    """A slab on the library: the solver, plus device buffers for the cuts."""

    def __init__(self, mask: np.ndarray, lo: int, hi: int, tau: float, drho: float, options=None):
        import torch

        from . import lbm
        self._lbm = lbm
        self._torch = torch
        x0, _, ghosts = slab_extent(lo, hi, mask.shape[-1])
        if options is None:
            options = lbm.make_options(stream=torch.cuda.current_stream().cuda_stream)
        self.solver = lbm.lbm_slab_create(slab_mask(mask, lo, hi), tau, drho, x0, mask.shape[-1], ghosts, options)
        self.ghosts = ghosts

    def step(self, n: int) -> None:
        self._lbm.lbm_step(self.solver, n)

    def halo_floats(self, side: int, incoming: bool = False) -> int:
        return self._lbm.lbm_slab_halo_floats(self.solver, side, incoming)

    def new_buffer(self, n: int):
        return self._torch.empty(n, dtype=self._torch.float32, device="cuda")

    def export(self, side: int, buf) -> None:
        self._lbm.lbm_slab_export(self.solver, side, buf)

    def import_(self, side: int, buf) -> None:
        self._lbm.lbm_slab_import(self.solver, side, buf)

    def observe(self) -> np.ndarray:
        return self._lbm.lbm_step_observe(self.solver, 0)[0]

    def finalize(self, obs_sum: np.ndarray):
        return self._lbm.lbm_slab_observables(self.solver, obs_sum)

    def close(self) -> None:
        self.solver.close()


class SlabDriver:
    """Advance a domain's slabs with the halo exchange after every step.

    slabs: this process's slabs, consecutive, the first being slab number
    `first` of `total`; group/ranks: the process group and, per slab number,
    the rank holding it (None: every slab is here)."""

    def __init__(self, slabs: Sequence, first: int, total: int, owner: Optional[Sequence[int]] = None,
                 dist=None, group=None, sync=None):
        self.slabs = list(slabs)
        self.first = first
        self.total = total
        self.owner = list(owner) if owner is not None else [0] * total
        self.dist = dist
        self.group = group
        self.sync = sync  # called between the steps of the slabs and the exchange (e.g. a stream sync)
        self.rank = dist.get_rank(group) if dist is not None else 0
        self._send, self._recv = {}, {}
        for j, s in enumerate(self.slabs):
            g = first + j
            for side in (0, 1):
                nb = g - 1 if side == 0 else g + 1
                if 0 <= nb < total:
                    self._send[(g, side)] = s.new_buffer(s.halo_floats(side, False))
                    self._recv[(g, side)] = s.new_buffer(s.halo_floats(side, True))

    def _local(self, g: int) -> Optional[object]:
        j = g - self.first
        return self.slabs[j] if 0 <= j < len(self.slabs) else None

    def exchange(self) -> None:
        for j, s in enumerate(self.slabs):
            g = self.first + j
            for side in (0, 1):
                if (g, side) in self._send:
                    s.export(side, self._send[(g, side)])
        if self.sync is not None:
            self.sync()
        ops = []
        for j, s in enumerate(self.slabs):
            g = self.first + j
            for side in (0, 1):
                if (g, side) not in self._recv:
                    continue
                nb, nb_side = (g - 1, 1) if side == 0 else (g + 1, 0)
                if self._local(nb) is not None:
                    self._recv[(g, side)].copy_(self._send[(nb, nb_side)])
                else:
                    peer = self.owner[nb]
                    ops.append(self.dist.P2POp(self.dist.isend, self._send[(g, side)], peer, self.group))
                    ops.append(self.dist.P2POp(self.dist.irecv, self._recv[(g, side)], peer, self.group))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        for j, s in enumerate(self.slabs):
            g = self.first + j
            for side in (0, 1):
                if (g, side) in self._recv:
                    s.import_(side, self._recv[(g, side)])

    def step(self, n: int) -> None:
        for _ in range(n):
            for s in self.slabs:
                s.step(1)
            self.exchange()

    def observe(self):
        """(k, Kn, residual) of the whole domain: observables of every slab,
        summed here and over the process group (slot 3: maximum)."""
        obs = np.zeros(8)
        for s in self.slabs:
            o = np.asarray(s.observe(), np.float64)
            obs[3] = max(obs[3], o[3])
            mask = np.ones(8, bool)
            mask[3] = False
            obs[mask] += o[mask]
        if self.dist is not None:
            import torch
            dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
            t = torch.tensor(obs, dtype=torch.float64, device=dev)
            m = torch.tensor([obs[3]], dtype=torch.float64, device=dev)
            self.dist.all_reduce(t, group=self.group)
            self.dist.all_reduce(m, op=self.dist.ReduceOp.MAX, group=self.group)
            obs = t.cpu().numpy().copy()
            obs[3] = float(m[0])
        return self.slabs[0].finalize(obs)
