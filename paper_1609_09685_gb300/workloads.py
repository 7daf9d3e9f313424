"""Seeded synthetic workloads shaped like the paper's experiments (Sec. 2).

This module only chooses inputs -- sizes, porosities, relaxation times,
pressure differences and seeds -- and holds none of the method's arithmetic.
Both the CUDA path and the oracle draw their inputs from here.  The paper's
own geometries (its 2D quartet structure and 3D sample) are not published with
it; seeded QSGS masks at the stated sizes and porosities stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

# Sec. 2: resolutions and porosities of the 2D tau sweep.
SWEEP_SIZES = [(400, 200, 0.7394), (800, 400, 0.7532), (1200, 600, 0.7578)]
# tau - 1/2 values of the sweep.
SWEEP_TAU_MINUS_HALF = [0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 1.5]
CORE_P = 0.02
D_FACE = 0.2


@dataclass
class Domain:
    nx: int
    ny: int
    nz: int
    porosity: float
    seed: int
    tau: float
    drho: float
    core_p: float = CORE_P
    d_face: float = D_FACE

    @property
    def shape(self):
        return (self.ny, self.nx) if self.nz == 1 else (self.nz, self.ny, self.nx)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz


@dataclass
class Workload:
    name: str
    domains: List[Domain] = field(default_factory=list)
    rho_out: float = 1.0
    tol: float = 1e-9
    max_steps: int = 20000

    @property
    def cells(self):
        return sum(d.cells for d in self.domains)


def stokes_drho(tau: float, nx: int) -> float:
    """Pressure difference (as a density difference) small enough for Stokes
    flow at every tau of the sweeps: min(1e-3, 1e-4 (tau - 1/2)/3 (nx - 1))."""
    return min(1e-3, 1e-4 * (tau - 0.5) / 3.0 * (nx - 1))


def small_2d(seed: int = 1) -> Workload:
    """100 x 50 D2Q9, QSGS core probability 0.02 to porosity 0.74, tau = 0.8,
    rho_in / rho_out = 1.0005 / 1.0, residual 1e-9 or 20000 steps."""
    return Workload("d2q9_100x50_tau0.8", [Domain(100, 50, 1, 0.74, seed, 0.8, 0.0005)],
                    tol=1e-9, max_steps=20000)


def tau_sweep(sizes=None, taus=None, seed: int = 1) -> Workload:
    """The Sec. 2 sweep: every (resolution, tau) pair as one domain of a batch
    (24 domains: 3 resolutions x 8 relaxation times), one mask per resolution."""
    sizes = SWEEP_SIZES if sizes is None else sizes
    taus = [0.5 + t for t in (SWEEP_TAU_MINUS_HALF if taus is None else taus)]
    doms = []
    for nx, ny, phi in sizes:
        for tau in taus:
            doms.append(Domain(nx, ny, 1, phi, seed, tau, stokes_drho(tau, nx)))
    return Workload("d2q9_tau_sweep_400x200_800x400_1200x600", doms, tol=1e-9, max_steps=10**7)


def batch128(master_seed: int = 2026, n: int = 128) -> Workload:
    """128 independent uneven D2Q9 domains: nx uniform over the even numbers in
    [200, 1200], ny = nx/2, porosity U[0.6, 0.8], tau U[0.51, 1.5], own seeds."""
    rng = np.random.default_rng(master_seed)
    doms = []
    for _ in range(n):
        nx = 2 * int(rng.integers(100, 601))
        phi = float(rng.uniform(0.6, 0.8))
        tau = float(rng.uniform(0.51, 1.5))
        seed = int(rng.integers(1, 2**62))
        doms.append(Domain(nx, nx // 2, 1, phi, seed, tau, stokes_drho(tau, nx)))
    return Workload("d2q9_batch128_uneven", doms, tol=1e-9, max_steps=10**7)


def d3q19_256(taus=(0.52, 0.6, 0.8, 1.0), seed: int = 1) -> Workload:
    """256 x 128 x 128 D3Q19, 3D QSGS to porosity 0.70, one domain per tau."""
    return Workload("d3q19_256x128x128", [Domain(256, 128, 128, 0.70, seed, t, stokes_drho(t, 256))
                                          for t in taus], tol=1e-9, max_steps=10**7)
