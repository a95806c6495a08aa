"""GB300-native ChebFD: the block Chebyshev polynomial filter of arxiv 1803.02156
(Kreutzer et al.) as hand-written sm_103a CUDA kernels behind a C ABI
(include/cfd.h, libcfd.so), with a thin ctypes binding.

Submodules:
  binding    ctypes binding of libcfd.so (same names as the C ABI)
  build      in-tree nvcc build of libcfd.so
  inputs     seeded synthetic inputs (SplitMix64), no method arithmetic
  workloads  named lattice / search-space configurations
  model      minimum-traffic and flop model of a filter step (Eq. 2)

Importing the package does not load the CUDA library; the first binding call
does, and raises if it is missing.
"""
__version__ = "1.0.0"
