"""GB300-native checkerboard Metropolis and population annealing (arXiv:1709.04394).

``gbmc``: ctypes binding of the C-ABI CUDA library ``libgbmc.so`` (built by
``build.build()``); ``exact``: exact finite-lattice 2D Ising results;
``inputs``: seeded synthetic workloads.
"""
from . import exact  # noqa: F401
