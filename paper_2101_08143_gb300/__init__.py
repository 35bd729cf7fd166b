"""GB300 (sm_103a) solver for the Friedkin-Johnsen opinion-dynamics quantities
of Xu, Bao and Zhang, "Fast Evaluation for Relevant Quantities of Opinion
Dynamics" (WWW 2021).

Submodules:
  fj     ctypes binding of libfj.so (the C ABI in include/fj.h)
  synth  seeded synthetic graphs and opinion vectors
  build  nvcc build of libfj.so for sm_103a

The binding loads the CUDA library on first use; there is no CPU fallback.
"""
__all__ = ["fj", "synth", "build"]
