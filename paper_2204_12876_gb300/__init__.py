"""GB300 (sm_103a) elevation-map fusion: point clouds into a robot-centric 2.5D
height grid, after Miki et al., arXiv 2204.12876, Section II.

The compute path is libem.so (hand-written CUDA kernels behind the C ABI of
include/em.h); ``em`` is its ctypes binding.  Build with ``build.build()``.
"""
from . import build  # noqa: F401
