"""RAM (Rapid Advection Algorithm on Arbitrary Meshes) on GB300.

The compute path is the CUDA library ``libram_gb300.so`` behind the C ABI in
``include/ram.h``; ``paper_2305_05362_gb300.ram`` is its thin ctypes binding.
Importing this package does not load the library; ``ram`` loads it on first
use and raises if it is missing.
"""
__all__ = ["ram", "workloads"]
