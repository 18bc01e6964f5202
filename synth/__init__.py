"""Seeded synthetic input generators (no arithmetic of the method itself).

Shared by the FP64 oracle tests and by the CUDA path's tests and benchmark.
"""
from .philox import philox4x32_10, uniform24, uniform53  # noqa: F401
from .matrices import *  # noqa: F401,F403
