"""GB300 (sm_103a) library for the Galilean-invariant preconditioned cascaded
central-moment lattice Boltzmann method on D2Q9 (arXiv 1806.10251).

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); :mod:`.lbm` is its ctypes binding.
"""
from .lbm import (GI_CUBIC_ONLY, GI_FULL, GI_UNCORRECTED, STORAGE_BF16, STORAGE_F16, STORAGE_F32,
                  STORAGE_F64, LbmError, Solver, lib, solver_from_case, use_torch_allocator)

__all__ = ["Solver", "LbmError", "lib", "solver_from_case", "use_torch_allocator", "GI_UNCORRECTED",
           "GI_CUBIC_ONLY", "GI_FULL", "STORAGE_F32", "STORAGE_F16", "STORAGE_BF16", "STORAGE_F64"]
