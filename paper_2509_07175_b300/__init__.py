"""B300-native clipped / restricted Voronoi diagrams by point-in-cell tests.

The compute path is ``libvd.so`` (hand-written CUDA for sm_103a, C ABI in
``include/vd.h``); ``binding`` is a thin ctypes layer over it that takes and
returns torch CUDA tensors.  ``inputs`` holds the seeded workload generators,
``parallel`` the partition of one diagram across ranks (host routing of pair
keys and moved sites), ``learned`` the training driver of the learned
proposal's network and ``serial`` the paper's serial method on the CPU.
"""
import importlib

from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "build", "parallel", "learned", "serial"]


def __getattr__(name):
    if name in ("binding", "build", "parallel", "learned", "serial"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
