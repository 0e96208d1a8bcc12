"""GB300-native line-of-sight projection (arXiv 2509.25110, Eqs. 1-2).

Submodules:
  gcamb  -- ctypes binding of libgcamb.so (the C ABI in include/gcamb.h)
  synth  -- seeded synthetic inputs (grids, sources, primordial spectrum)
  build  -- nvcc build of libgcamb.so for sm_103a

Importing the package loads nothing; the library is loaded on first use.
"""
__all__ = ["gcamb", "synth", "build"]
