"""GB300-native harmonic-balance residual library (libhb.so) and its Python binding.

``cases`` generates seeded synthetic workloads; ``hb`` binds the C ABI of
``include/hb.h``; ``build`` compiles the CUDA library for sm_103a.
"""
from . import cases  # noqa: F401

__all__ = ["cases", "hb", "build"]
