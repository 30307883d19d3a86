"""B300-native clipped / restricted Voronoi diagrams by point-in-cell tests.

The compute path is ``libvd.so`` (hand-written CUDA for sm_103a, C ABI in
``include/vd.h``); ``binding`` is a thin ctypes layer over it that takes and
returns torch CUDA tensors.  ``inputs`` holds the seeded workload generators.
"""
import importlib

from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "build"]


def __getattr__(name):
    if name in ("binding", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
