"""GB300-native lattice-Boltzmann sweep with the single-node second-order boundary
schemes of Zhao & Yong (arXiv:1712.08288).

The computation lives in the CUDA library liblbm.so (C-ABI: include/lbm.h); the
``binding`` module is a ctypes wrapper with the same call names, and ``workloads``
generates seeded synthetic inputs (geometries, wall fractions, wall velocities).
"""

__all__ = ["binding", "workloads"]
