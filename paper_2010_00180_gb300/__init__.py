"""GB300-native quantum-inspired search for low-energy states of Ising Hamiltonians.

Submodules:
  inputs  -- seeded synthetic instances and initial states (no method arithmetic)
  qis     -- ctypes binding of the CUDA library libqis.so (the C-ABI in include/qis.h)
  build   -- nvcc build of libqis.so for sm_103a
"""
