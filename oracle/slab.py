"""An x-slab of a domain stepped by the FP64 oracle -- TEST INFRASTRUCTURE ONLY.

The slab holds its real columns [lo, hi) of the whole domain plus a ghost
column at each cut (a copy of the neighbouring slab's edge column).  One step
is the oracle's own step (`oracle.step`) on that extended array: every real
node pulls from the ghost exactly what it would pull from the neighbour's
column in the whole domain, so after the ghosts are refreshed the real columns
equal the whole domain's, bit for bit.  The ghosts' own results (the step also
applies its x-face boundaries to them) are discarded: the next exchange
overwrites them.  The exchange carries, per cut, the planes whose direction
crosses it (c_x = -1 leftwards, +1 rightwards) of the fluid nodes of one
column, in (z, y) order, as a float64 buffer.

It implements the slab interface of the library's slab driver (step,
halo_floats, new_buffer, export, import_, observe, finalize) so that the
driver's exchange logic runs on CPU ranks; it shares no code with it.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


class OracleSlab:
    def __init__(self, mask, lo, hi, tau, drho, rho_out=1.0, eq=O.EQ_QUADRATIC):
        mask = np.ascontiguousarray(mask, np.uint8)
        nx = mask.shape[-1]
        self.lo, self.hi, self.nx = lo, hi, nx
        self.left = 1 if lo > 0 else 0
        self.right = 1 if hi < nx else 0
        self.x0 = lo - self.left
        self.mask = np.ascontiguousarray(mask[..., self.x0:hi + self.right])
        self.tau, self.drho, self.rho_out, self.eq = tau, drho, rho_out, eq
        self.q = 9 if mask.ndim == 2 else 19
        c = O.lattice(self.q)[0]
        self.planes = {-1: [i for i in range(self.q) if c[i][0] == -1], 1: [i for i in range(self.q) if c[i][0] == 1]}
        # the whole domain's initial state, cut to the slab (ghosts included)
        self.f = np.ascontiguousarray(O.init(mask, 1.0 + drho, rho_out)[..., self.x0:hi + self.right, :])

    # columns of the extended array
    def _col(self, which):
        n = self.mask.shape[-1]
        return {"first": self.left, "last": n - 1 - self.right, "lghost": 0, "rghost": n - 1}[which]

    def _fluid(self, x):
        return self.mask[..., x] == 0

    def step(self, n):
        for _ in range(n):
            self.f = O.step(self.mask, self.f, self.tau, 1.0 + self.drho, self.rho_out, self.eq)

    def halo_floats(self, side, incoming=False):
        if incoming:
            x = self._col("lghost" if side == 0 else "rghost")
            return len(self.planes[1 if side == 0 else -1]) * int(self._fluid(x).sum())
        x = self._col("first" if side == 0 else "last")
        return len(self.planes[-1 if side == 0 else 1]) * int(self._fluid(x).sum())

    def new_buffer(self, n):
        import torch
        return torch.zeros(n, dtype=torch.float64)

    def export(self, side, buf):
        x = self._col("first" if side == 0 else "last")
        col = self.f[..., x, :][self._fluid(x)]  # (fluid nodes in (z, y) order, Q)
        buf.numpy()[:] = col[:, self.planes[-1 if side == 0 else 1]].T.ravel()

    def import_(self, side, buf):
        x = self._col("lghost" if side == 0 else "rghost")
        fl = self._fluid(x)
        p = self.planes[1 if side == 0 else -1]
        vals = buf.numpy().reshape(len(p), int(fl.sum())).T
        col = self.f[..., x, :]
        sub = col[fl]
        sub[:, p] = vals
        col[fl] = sub
        self.f[..., x, :] = col

    def real(self):
        """The slab's real columns of the populations."""
        n = self.mask.shape[-1]
        return self.f[..., self.left:n - self.right, :]

    def observe(self):
        """Slot 0: the link flux of the planes x + 1/2 with x a real column
        (the right cut's plane included: its ghost holds the neighbour's column
        after an exchange); the other slots are left at zero."""
        J = O.link_flux(self.mask, self.f)
        n = self.mask.shape[-1]
        last = n - 1 - self.right
        out = np.zeros(8)
        out[0] = J[self.left:min(last + 1, n - 1)].sum()
        return out

    def finalize(self, obs_sum):
        """Darcy's law with the summed link flux (the oracle's permeability,
        Sec. 2; nu = (tau - 1/2)/3, Eq. 1) over the whole domain; Kn and the
        residual are not formed here."""
        ny = self.mask.shape[-2]
        nz = self.mask.shape[0] if self.mask.ndim == 3 else 1
        nu = (self.tau - 0.5) / 3.0
        return nu * obs_sum[0] / (ny * nz / 3.0 * self.drho), None, None
