"""GB300-native spherical harmonic transforms (Reinecke & Seljebotn 2013, libsharp).

Submodules:
  sht     -- ctypes binding of the C-ABI library ``libsht_gb300.so`` (the CUDA path)
  build   -- compiles that library for sm_103a with nvcc
  inputs  -- seeded synthetic a_lm / map generators (no transform arithmetic)
  autograd -- torch.autograd.Function wrappers over the C-ABI

Importing the package loads nothing; ``from paper_1303_4945_gb300 import sht``
loads the CUDA library and raises if it is missing.
"""
