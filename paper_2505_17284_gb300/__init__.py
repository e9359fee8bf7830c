"""GB300 (sm_103a) explicit S_N transport step for the lattice and enclosure benchmarks.

The compute path is librt_gb300.so (CUDA kernels behind the C ABI of
include/rt.h); `rt` is its thin Python binding. `build.build()` compiles it.
"""
from . import rt  # noqa: F401

__all__ = ["rt"]
