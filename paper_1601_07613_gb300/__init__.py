"""Colored, race-free DG right-hand side for GB300 (sm_103a).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/dgc.h``); ``dgc`` is its ctypes binding and ``workloads`` the seeded
synthetic input generators.  Importing the package does not load the library;
``dgc.lib()`` does, and raises if it cannot be built or loaded.
"""

__all__ = ["dgc", "workloads"]
