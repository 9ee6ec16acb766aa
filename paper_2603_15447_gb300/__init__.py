"""GB300-native batched Bezier / B-spline / NURBS / surface evaluation.

The compute path is libbez.so (hand-written sm_103a CUDA kernels behind the C
ABI in include/bez.h); ``bez`` is its thin ctypes binding and ``synth`` the
seeded input generator.  Importing the package does not load the library;
the first call does, and raises if it has not been built.
"""
import importlib

from . import synth  # noqa: F401

__all__ = ["bez", "synth"]


def __getattr__(name):
    if name in ("bez", "build", "autograd"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
