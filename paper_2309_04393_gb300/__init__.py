"""Residency-octree ray caster for GB300 (sm_103a).

The compute path lives in libro.so (CUDA kernels behind the C ABI of
include/ro.h); `ro` is its ctypes binding.
"""
from . import build, ro  # noqa: F401

__all__ = ["build", "ro"]
