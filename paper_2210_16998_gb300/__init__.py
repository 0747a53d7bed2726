"""GB300-native prime-path and test-path generation (TPGen hot path).

Submodules:
  cfggen -- seeded synthetic control-flow graphs (inputs only)
  build  -- nvcc build of libtpg.so for sm_103a
  tpg    -- ctypes binding of the C ABI in include/tpg.h

Importing the package loads nothing; ``tpg.load_library()`` (called by every
binding function) loads the CUDA library and raises if it is missing.
"""
