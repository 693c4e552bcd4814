"""B300-native (sm_103a) finite-volume Euler solver of arXiv:2512.13403 behind a C ABI.

The compute path is the CUDA library libdh.so (include/dh.h); ``solver.Solver`` marshals
arguments to it.  ``inputs`` builds seeded synthetic initial conditions.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "solver", "build"]
