"""GB300-native two-component D3Q19 lattice-Boltzmann (Shan-Chen) solver.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lb.h``); this package only marshals arguments to it. Importing the
package does not load the library; constructing a ``Solver`` does, and fails
loudly when it has not been built.
"""
from .single import SingleFluid  # noqa: F401
from .solver import Solver, create, run_host  # noqa: F401

__all__ = ["Solver", "SingleFluid", "create", "run_host"]
