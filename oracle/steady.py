"""Steady state of the oracle's step as a fixed point -- TEST INFRASTRUCTURE ONLY.

Sec. 2 iterates the lattice Boltzmann step "to steady state".  For a
percolating mask that state is the unique fixed point f* = S(f*) of the step
map S (stream, Zou-He, collide), and the permeability is Darcy's law applied to
f*.  Iterating S converges geometrically, but on the paper's larger domains the
slowest pressure mode takes 10^5 - 10^6 steps, far beyond what a plain FP64 CPU
step can do in a test budget.  This module finds the same fixed point by
solving F(x) = S(x) - x = 0 with a Newton-Krylov method (scipy's
`newton_krylov`, LGMRES inner solves, Jacobian-vector products by finite
differences of S): a library root finder used as the "iterate to steady
state" step.  Every evaluation of S is one call of the oracle's own FP64 step
(`oracle.step`), so the state it returns is a fixed point of exactly the
oracle's arithmetic.  What it adds is checked in the CPU tests: on small
domains it equals the plain iteration's converged state, and on the straight
channel it reproduces the exact discrete solution.

Only the test-suite, the golden-value script under tests/golden/ and the
benchmark's baseline legs use it.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def _pack_maps(mask):
    m = np.ascontiguousarray(mask, np.uint8)
    q = 9 if m.ndim == 2 else 19
    fluid = m == 0
    return m, q, fluid, int(fluid.sum())


def steady_state(mask, tau, rho_in, rho_out, eq=O.EQ_QUADRATIC, tau_m=None, f0=None, f_tol=4e-16,
                 inner_maxiter=30, maxiter=400, verbose=False):
    """Fixed point of the oracle step for a pressure-driven domain.

    Unknowns are the fluid nodes' populations shifted by w_i rho_out (their
    deviation from the rest state at the outlet density).  Starts from f0, or
    from the linear-ramp rest equilibrium of the solver's own initial state.
    Returns (f, info): f dense unshifted populations; info the max-norm of
    S(f) - f, the number of step evaluations and whether the root finder met
    f_tol."""
    from scipy.optimize import newton_krylov
    from scipy.optimize import NoConvergence

    m, q, fluid, nf = _pack_maps(mask)
    w = O.lattice(q)[1]
    shape = m.shape + (q,)

    def unpack(x):
        f = np.zeros(shape)
        f[fluid] = x.reshape(nf, q) + w * rho_out
        return f

    def pack(f):
        return (f[fluid] - w * rho_out).ravel()

    evals = [0]

    def F(x):
        evals[0] += 1
        return pack(O.step(m, unpack(x), tau, rho_in, rho_out, eq, tau_m)) - x

    x0 = pack(O.init(m, rho_in, rho_out) if f0 is None else f0)
    converged = True
    try:
        x = newton_krylov(F, x0, method="lgmres", inner_maxiter=inner_maxiter, f_tol=f_tol, maxiter=maxiter,
                          verbose=verbose)
    except NoConvergence as e:  # keep the best iterate; its residual is reported
        x = e.args[0]
        converged = False
    r = float(np.abs(F(x)).max())
    return unpack(x), {"residual_max": r, "evaluations": evals[0], "converged": converged}
