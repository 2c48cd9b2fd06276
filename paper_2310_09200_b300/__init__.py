"""B300-native Bluebild standard synthesis (BIPP, arXiv:2310.09200).

Submodules:
  inputs   — seeded synthetic data (layouts, skies, visibilities, pixel grids)
  bipp_ss  — ctypes binding of the C-ABI library ``libbipp_ss.so``
  build    — nvcc build of the CUDA library for sm_103a

The CUDA library is loaded lazily by ``bipp_ss``; importing the package does
not touch the GPU.
"""
__all__ = ["inputs", "bipp_ss", "build"]
