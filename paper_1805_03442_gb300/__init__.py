"""GB300-native solver for unstable sound waves in a vibrationally excited gas
(Khrapov & Khoperskov 2018): the MUSCL-Hancock finite-volume step of Sec. 2.3
as fused CUDA kernels behind the C-ABI library ``libsv.so``.

Submodules:
  ``sv``      -- ctypes binding of libsv.so (Solver, Batch); raises if the
                 library is missing, there is no CPU fallback.
  ``build``   -- nvcc build of libsv.so for sm_103a, in-tree.
  ``inputs``  -- seeded synthetic initial states (no method arithmetic).
"""
__all__ = ["sv", "build", "inputs"]
