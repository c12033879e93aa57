"""GB300 (sm_103a) multiscale-multigrid heat solver for SIMP topology
optimisation (arXiv 2410.06850), exposed through the C ABI in include/thermo.h.

Modules
  thermo    ctypes binding of libthermo.so (same entry-point names)
  autograd  torch.autograd.Function wrappers: compliance and density filter
  build     in-tree nvcc build of libthermo.so
"""
from .thermo import (FP64, MIXED, MIXED_BF16S, PC_MMG, PC_NONE, PC_JACOBI,  # noqa: F401
                     GUESS_ZERO, GUESS_GIVEN, GUESS_COARSE, GUESS_WARM_COARSE,
                     Solver, ThermoError, default_options, lib)
