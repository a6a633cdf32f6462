"""GB300-native periodic Ewald summation for quantum Monte Carlo walkers.

The compute path is the C-ABI library ``libewald_gb300.so`` (hand-written
CUDA kernels for sm_103a); ``paper_2507_02888_gb300.ewald`` is its thin
Python binding.  Importing the package itself loads nothing.
"""
__all__ = ["ewald", "inputs"]
