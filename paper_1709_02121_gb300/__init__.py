"""GB300 (sm_103a) signed-particle Wigner branching random walk.

The data-parallel hot path of Xiong & Shao, "The Wigner branching random walk:
efficient implementation and performance evaluation" (arXiv:1709.02121):
free streaming, branching on a counter-based Philox clock, +/- pair spawning,
offspring compaction, and resampling by annihilation (sp1) or by the signed
bootstrap filter (sp2).  All of it runs in hand-written CUDA kernels behind
the C ABI of include/wbrw.h; ``wbrw`` is its ctypes binding.
"""
from . import grad, wbrw  # noqa: F401
from .wbrw import Batch, Simulation, Simulation4, WbrwError, load  # noqa: F401

__all__ = ["grad", "wbrw", "Batch", "Simulation", "Simulation4", "WbrwError", "load"]
