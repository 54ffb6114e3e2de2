"""B300 (sm_103a) implementation of the data-parallel hot path of HALLaR.

Submodules:
  hallar     ctypes binding of the C ABI (include/hallar.h); loads libhallar.so
  build      nvcc build of libhallar.so from csrc/
  instances  seeded synthetic SDP instances (input data only)

Importing the package loads nothing; ``from paper_2505_13719_b300 import hallar``
loads the CUDA library and raises if it is missing.
"""
