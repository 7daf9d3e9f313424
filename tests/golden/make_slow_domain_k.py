"""Writes slow_domain_k.txt: the FP64 oracle's permeability of one 512x256
QSGS domain whose slowest pressure mode relaxes over ~5e4 steps, after exactly
250000 steps from the equilibrium start (the oracle's own k changes by < 1e-6
relative after that).  Calls only oracle/.  Takes about an hour on one core:

    python tests/golden/make_slow_domain_k.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

SHAPE = (256, 512)
SEED, CORE_P, PHI = 1000006, 0.02, 0.621370254804748
TAU, DRHO = 0.7653754091733804, 1e-3
STEPS = 250_000


def main():
    mask, it = O.qsgs(SHAPE, SEED, CORE_P, PHI)
    f = O.init(mask, 1 + DRHO, 1.0)
    f = O.run(mask, f, TAU, 1 + DRHO, 1.0, STEPS)
    k = O.permeability(mask, f, TAU, 1 + DRHO, 1.0)
    with open(os.path.join(HERE, "slow_domain_k.txt"), "w") as fh:
        fh.write("# FP64 oracle, written by make_slow_domain_k.py: QSGS (ny, nx) = (256, 512), seed 1000006,\n")
        fh.write("# core_p 0.02, porosity 0.621370254804748, tau 0.7653754091733804, drho 1e-3,\n")
        fh.write("# equilibrium start (linear density ramp), 250000 steps; then k (lattice units^2)\n")
        fh.write(f"steps {STEPS}\nk {k:.15e}\n")


if __name__ == "__main__":
    main()
