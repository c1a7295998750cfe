"""GB300-native per-point rank-one convexification (arXiv 2211.14318).

The compute path is libconvexify.so (hand-written CUDA for sm_103a, C ABI in
include/convexify.h); ``api`` is its Python binding and ``inputs`` the seeded
synthetic workloads.  Importing the package does not load the library.
"""
__all__ = ["api", "inputs", "build"]
