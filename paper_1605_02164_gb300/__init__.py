"""GB300 (sm_103a) Monte Carlo shiftable bilateral filter for vector-valued
images (Ghosh & Chaudhury, arXiv 1605.02164).

The compute path is the CUDA library libbf (C ABI in include/bf.h); ``bf``
is its ctypes binding, ``synth`` draws seeded synthetic inputs, ``serve``
runs the batched request loop.  Importing the package does not load the
library; the first call into ``bf`` does, and fails if it is not built.
"""
__all__ = ["bf", "synth", "build"]
__version__ = "1.0.0"
