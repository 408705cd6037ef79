"""GB300-native fast finite-difference solver for 3D Helmholtz problems in layered media.

The solver (block-wise separable eigen-transform solve in x/y, tridiagonal
solves in z per mode, and the interface correction of Sec. 2) lives in the
CUDA library built from `csrc/`; `hz` is its thin Python binding.  Importing
the package does not load the library: `from paper_1909_01299_gb300 import hz`
does, and fails loudly when it is missing.
"""
__all__ = ["hz", "workloads", "build"]
