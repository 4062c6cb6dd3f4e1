"""GB300 (sm_103a) implementation of the entropy-stable van der Waals moving-mesh scheme.

Submodules
  es        -- ctypes binding of the C-ABI library ``libesvdw.so`` (the compute path)
  build     -- compiles the CUDA library for sm_103a with nvcc
  workloads -- seeded synthetic inputs (primitive fields and meshes only)

Importing the package loads nothing; ``es`` loads the CUDA library on first use
and raises if it is missing.
"""
