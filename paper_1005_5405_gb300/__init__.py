"""GB300-native semi-regular Boltzmann solver (driven cavity, hard spheres).

The numerical method is that of Frezzotti, Ghiroldi & Gibelli, "Solving the
Boltzmann equation on GPUs": first-order upwind free streaming with Maxwell
diffuse walls, a Monte Carlo evaluation of the hard-sphere collision integral
on a Cartesian velocity grid, and the Aristov-Tcheremissine conservation
correction.  Every step runs in hand-written sm_103a CUDA kernels behind the
C ABI declared in include/bz.h; this package is a thin ctypes binding.
"""
from .workloads import Problem  # noqa: F401

__all__ = ["Problem"]
