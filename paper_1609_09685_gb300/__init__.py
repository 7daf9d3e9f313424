"""GB300-native lattice Boltzmann permeability library (arXiv:1609.09685).

``lbm`` is the ctypes binding of the C ABI in ``include/lbm.h``; ``build``
compiles the CUDA library in-tree; ``workloads`` holds the seeded synthetic
inputs shaped like the paper's experiments.
"""
__all__ = ["lbm", "build", "workloads"]
