"""GB300-native Friedkin-Johnsen equilibrium solver (local residual push, SOR, FP64 certificate).

The compute lives in ``libfj.so`` (CUDA kernels for sm_103a behind the C ABI of
``include/fj.h``); ``paper_2507_14864_gb300.capi`` is its thin Python binding.
``build()`` compiles the library.
"""
from .buildlib import build  # noqa: F401

__all__ = ["build"]
