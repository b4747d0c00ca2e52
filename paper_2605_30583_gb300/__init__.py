"""GB300-native Levenberg-Marquardt + PCGNR bundle adjustment (arXiv 2605.30583, Caspar).

The solver lives in libgbba.so (hand-written CUDA for sm_103a behind a C ABI,
include/gbba.h); `binding` is its ctypes wrapper, `autograd` the torch.autograd
Function over the reprojection cost, `synth` the seeded synthetic workloads.
Importing the package loads nothing; the library is loaded on first use and a
missing build raises an error.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "binding"]
