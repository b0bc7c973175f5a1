"""GB300-native Metropolis SA / PT for tile-planted cubic-lattice Ising spin glasses.

The compute path lives in the CUDA library ``libsg.so`` (C ABI declared in
``include/sg.h``); ``paper_2501_17267_gb300.sg`` is its thin ctypes binding.
Importing the package does not load the library; importing ``.sg`` does, and
raises if the library has not been built.
"""
__all__ = ["sg", "workloads"]
