"""GB300-native arc-length WENO (WENO-L) solver for Hamilton-Jacobi equations.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/alweno.h``); ``native`` is its Python binding and ``inputs`` holds
the seeded synthetic workloads.  Importing this package does not load the
library; creating a solver does, and fails loudly if it is missing.
"""
__all__ = ["native", "inputs", "build"]
