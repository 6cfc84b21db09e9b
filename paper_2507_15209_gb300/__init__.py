"""GB300 (sm_103a) implementation of the in-situ multipole 3PCF hot path of
Ju et al. (2025), arXiv:2507.15209.

Submodules:
  zeta      -- ctypes binding of libzeta (include/zeta.h); no arithmetic in Python
  build     -- nvcc build of libzeta.so in-tree
  mocks     -- seeded log-normal mock catalogues (inputs only)
  workloads -- named workload parameters
Importing the package has no side effects; the library is loaded on first use.
"""
__all__ = ["zeta", "build", "mocks", "workloads"]
