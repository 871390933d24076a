"""GB300-native tile-based differentiable Gaussian-splatting rasterizer.

The compute path is libgs.so (hand-written sm_103a CUDA behind the C ABI in
include/gs.h); this package holds its build script, the ctypes binding and
the torch-facing wrappers.  Importing it does not touch the GPU.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "raster", "build"]
