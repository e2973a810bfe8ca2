"""GB300-native cyclic-symmetry optimal transport (arXiv 2311.13147).

The compute path is the C-ABI library ``libcyclicot.so`` (hand-written CUDA
for sm_103a, declared in ``include/cyclicot.h``); ``cyclicot`` is its thin
Python binding.  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "cyclicot"]
