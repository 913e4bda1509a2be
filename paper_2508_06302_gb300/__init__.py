"""GB300-native FSE-Shooting (arXiv 2508.06302) hot path.

Submodules:
  inputs  -- seeded synthetic finite-element workloads (no method arithmetic)
  fse     -- ctypes binding of the CUDA C-ABI library (include/fse.h)
  _build  -- in-tree nvcc build of the library for sm_103a
"""
__all__ = ["inputs", "fse"]
