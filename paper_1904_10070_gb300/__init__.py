"""GB300-native vielbein lattice-Boltzmann + Cahn-Hilliard solver (arXiv:1904.10070).

Submodules:
  vlb     -- ctypes binding of the C ABI in include/vlb.h (libvlb.so, built by ``build``)
  inputs  -- seeded synthetic initial conditions and workload recipes
  build   -- nvcc build of libvlb.so for sm_103a
"""
