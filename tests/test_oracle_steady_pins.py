"""Pins of the oracle's fixed-point solver (oracle/steady.py), CPU only.

The solver finds the steady state of the oracle's own FP64 step with a
Newton-Krylov root finder instead of by iterating the step.  It is tied here to
things it must reproduce: the plain iteration's converged state on domains
small enough to iterate, and the exact discrete channel solution (a closed
form, derived independently of both)."""
import numpy as np
import pytest

import oracle as O
from oracle import steady

pytest.importorskip("scipy")


def _exact_channel_k(h, tau):
    # exact steady BGK channel with halfway bounce-back and the linear
    # equilibrium (derivation in test_oracle_pins._channel_exact_k)
    return (h * h - 1 + 8 * (tau - 0.5) ** 2) / 12.0


@pytest.mark.parametrize("eq", [O.EQ_QUADRATIC, O.EQ_LINEAR])
def test_fixed_point_equals_the_plain_iteration(eq):
    mask, _ = O.qsgs((20, 40), 3, 0.02, 0.72)
    assert O.percolates(mask)
    tau, drho = 0.9, 1e-3
    f_it, rc, _, _ = O.run_to_steady(mask, O.init(mask, 1 + drho, 1.0), tau, 1 + drho, 1.0, 1e-11, 2_000_000,
                                     eq=eq)
    assert rc == 0
    f_fp, info = steady.steady_state(mask, tau, 1 + drho, 1.0, eq=eq)
    assert info["converged"] and info["residual_max"] <= 4e-16
    # the plain iteration stalls at a rounding floor (its per-step change
    # stays ~1e-14, which the slow pressure modes turn into a ~1e-6 offset of
    # the density field); the root finder's state is the better fixed point
    r_it = np.abs(O.step(mask, f_it, tau, 1 + drho, 1.0, eq) - f_it).max()
    assert info["residual_max"] < r_it
    w = O.lattice(9)[1]
    fl = mask == 0
    dev = np.abs((f_it - w)[fl]).max()
    assert np.abs((f_fp - f_it)[fl]).max() <= 1e-5 * dev
    k_it = O.permeability(mask, f_it, tau, 1 + drho, 1.0)
    k_fp = O.permeability(mask, f_fp, tau, 1 + drho, 1.0)
    assert k_fp == pytest.approx(k_it, rel=1e-9)
    # further plain steps move k only by their own rounding floor
    f_more = O.run(mask, f_fp, tau, 1 + drho, 1.0, 50, eq)
    assert O.permeability(mask, f_more, tau, 1 + drho, 1.0) == pytest.approx(k_fp, rel=1e-10)


def test_fixed_point_reproduces_the_exact_channel_solution():
    h, tau = 10, 1.2
    ny, nx = h + 2, 6 * h
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    drho = 1e-3
    f, info = steady.steady_state(mask, tau, 1 + drho, 1.0, eq=O.EQ_LINEAR)
    assert info["converged"]
    rho, ux, _ = O.fields(mask, f)
    xm = nx // 2
    j = (rho * ux)[1:-1, xm]
    beta = (rho[1:-1, xm + h // 2] - rho[1:-1, xm - h // 2]).mean() / (2 * (h // 2))
    k_local = (tau - 0.5) / 3.0 * j.mean() / (-beta / 3.0)
    assert k_local == pytest.approx(_exact_channel_k(h, tau), rel=1e-9)


def test_fixed_point_from_another_start_is_the_same():
    """Uniqueness of the steady state (a percolating mask): starting from the
    rest state at the outlet density instead of the linear ramp gives the same
    fixed point."""
    mask, _ = O.qsgs((16, 32), 5, 0.02, 0.75)
    tau, drho = 0.7, 5e-4
    a, _ = steady.steady_state(mask, tau, 1 + drho, 1.0)
    b, _ = steady.steady_state(mask, tau, 1 + drho, 1.0, f0=O.init(mask, 1.0, 1.0))
    ka = O.permeability(mask, a, tau, 1 + drho, 1.0)
    kb = O.permeability(mask, b, tau, 1 + drho, 1.0)
    assert ka == pytest.approx(kb, rel=1e-10)


def test_a_state_at_the_residual_bound_fixes_k():
    """Stored oracle states are used when |S(f) - f| <= 1e-13.  On a 100x50
    benchmark domain a root-finder state stopped at that residual gives the
    permeability of the fully converged one (4e-16) to far better than the
    1e-4 the GPU comparison allows."""
    mask, _ = O.qsgs((50, 100), 1, 0.02, 0.74)
    tau, drho = 0.8, 5e-4
    f_lo, info_lo = steady.steady_state(mask, tau, 1 + drho, 1.0, f_tol=1e-13)
    f_hi, info_hi = steady.steady_state(mask, tau, 1 + drho, 1.0)
    assert info_lo["residual_max"] <= 1e-13 and info_hi["residual_max"] <= 4e-16
    k_lo = O.permeability(mask, f_lo, tau, 1 + drho, 1.0)
    k_hi = O.permeability(mask, f_hi, tau, 1 + drho, 1.0)
    assert k_lo == pytest.approx(k_hi, rel=1e-7)
