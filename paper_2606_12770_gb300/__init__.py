"""GB300-native state-vector simulator for the Carleman-linearised D1Q3
lattice-Boltzmann QSVT circuit (Kanno et al.).

The compute path is the C-ABI library ``_lib/libcsim.so`` (C++ host compiler
plus hand-written CUDA kernels for sm_103a); ``_native`` is its ctypes
binding.  Importing this package does not load the library; the first call
that needs it does, and raises if it cannot.
"""
from ._native import (CSIM_C64, CSIM_C128, CSIM_EXEC_FUSED, CSIM_EXEC_GATE, Circuit,  # noqa: F401
                      CsimError, Pool, StateVector, gates_to_records, load, pool_plan,
                      set_launch_shape)

__all__ = ["Circuit", "StateVector", "Pool", "pool_plan", "CsimError", "load", "gates_to_records",
           "set_launch_shape", "CSIM_C64",
           "CSIM_C128", "CSIM_EXEC_FUSED", "CSIM_EXEC_GATE"]
