"""GB300-native orthogonal discrete spherical Bessel transform (DSBT).

Submodules:
  dsbt    -- ctypes binding of the CUDA C-ABI library (loads libdsbt.so; raises if
             it is missing: there is no CPU fallback)
  inputs  -- seeded synthetic inputs (no transform arithmetic)
  build   -- nvcc build of the CUDA library
"""
__all__ = ["dsbt", "inputs", "build"]
