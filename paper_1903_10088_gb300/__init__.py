"""GB300-native OS-TV statistical iterative MVCT reconstruction (arXiv:1903.10088).

Submodules:
  ``mvct``    -- ctypes binding of the C-ABI CUDA library ``libmvct.so``
  ``phantom`` -- seeded synthetic inputs (ellipse phantoms, Poisson data)
  ``build``   -- compiles the CUDA library for sm_103a

Importing the package loads nothing; ``mvct`` raises if the library is missing.
"""
__all__ = ["mvct", "phantom", "build"]
