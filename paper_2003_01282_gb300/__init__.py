"""GB300-native stochastic Lanczos quadrature (SLaQ, WWW'20) for spectral
graph descriptors: NetLSD heat / wave traces and von Neumann graph entropy.

The computation lives in the CUDA library ``libslaq.so`` (C ABI in
``include/slaq.h``); :mod:`paper_2003_01282_gb300.slaq` is its ctypes
binding.  Build it with ``paper_2003_01282_gb300.build.build()``.
"""
from . import build, slaq  # noqa: F401

__all__ = ["slaq", "build"]
