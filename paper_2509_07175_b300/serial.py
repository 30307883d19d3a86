"""The paper's serial method (Alg. 1 + Alg. 2) on the CPU, single-threaded.

A CPU baseline of the method itself -- real edges, the breadth-first queue over
positive face flags, the intermediate polytope G_{a,j} -- built with gcc from
``serial/vd_serial.c``.  It shares no code with the GPU library or with the
oracle, and nothing on the GPU path calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "serial", "vd_serial.c")
_LIB = os.path.join(_HERE, "libvdserial.so")
STAT_NAMES = ("tests", "nn_queries", "clips", "g_clips", "bisector_faces", "excess_clips", "fallback",
              "fp128", "uncertain", "ties", "search_steps", "errors")


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [("np", ctypes.c_int64), ("a", ctypes.POINTER(ctypes.c_int32)),
                ("i", ctypes.POINTER(ctypes.c_int32)), ("meas", ctypes.POINTER(ctypes.c_double)),
                ("m1", ctypes.POINTER(ctypes.c_double)), ("foff", ctypes.POINTER(ctypes.c_int64)),
                ("flags", ctypes.POINTER(ctypes.c_int32)), ("fmeas", ctypes.POINTER(ctypes.c_double)),
                ("stats", ctypes.c_int64 * 12), ("status", ctypes.c_int)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.sv_create.restype = P
        lib.sv_create.argtypes = [ctypes.c_int, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, P]
        lib.sv_destroy.argtypes = [P]
        lib.sv_destroy.restype = None
        lib.sv_run.restype = ctypes.POINTER(_Result)
        lib.sv_run.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
        lib.sv_run_list.restype = ctypes.POINTER(_Result)
        lib.sv_run_list.argtypes = [P, P, ctypes.c_int64]
        lib.sv_free_result.argtypes = [ctypes.POINTER(_Result)]
        lib.sv_free_result.restype = None
        _lib = lib
    return _lib


class Pieces:
    """Every piece P_{a,i} the method produced: measure, first moment (frame of
    v_i), face flags of positive measure (Sec. 2.2), and the work counters."""

    def __init__(self, r: _Result):
        n = r.np
        take = lambda p, shape, dt: np.ctypeslib.as_array(p, shape).astype(dt) if n else np.zeros(shape, dt)  # noqa
        self.a = take(r.a, (n,), np.int64)
        self.i = take(r.i, (n,), np.int64)
        self.meas = take(r.meas, (n,), np.float64)
        self.m1 = take(r.m1, (n, 3), np.float64)
        self.foff = np.ctypeslib.as_array(r.foff, (n + 1,)).copy()
        nf = int(self.foff[-1])
        self.flags = np.ctypeslib.as_array(r.flags, (nf,)).copy() if nf else np.zeros(0, np.int32)
        self.fmeas = np.ctypeslib.as_array(r.fmeas, (nf,)).copy() if nf else np.zeros(0)
        self.stats = dict(zip(STAT_NAMES, list(r.stats)))
        self.status = int(r.status)

    def __len__(self):
        return len(self.a)

    def topology(self):
        """{(a, i): sorted face flags} over the pieces of positive measure."""
        out = {}
        for p in np.nonzero(self.meas > 0)[0]:
            out[(int(self.a[p]), int(self.i[p]))] = tuple(sorted(int(f) for f in
                                                                self.flags[self.foff[p]:self.foff[p + 1]]))
        return out


class Serial:
    """mode 2 (planar triangles, sites and vertices with z = 0), 3 (surface
    triangles in R^3), 4 (tetrahedra); sites (n, 3), verts (nv, 3) float64."""

    def __init__(self, mode, sites, verts, simp):
        self.sites = np.ascontiguousarray(sites, dtype=np.float64).reshape(-1, 3)
        self.verts = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3)
        self.simp = np.ascontiguousarray(simp, dtype=np.int32)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        self._h = _load().sv_create(int(mode), len(self.sites), p(self.sites), len(self.verts), p(self.verts),
                                    len(self.simp), p(self.simp))
        if not self._h:
            raise ValueError("invalid mesh (index out of range or a facet shared by more than two simplices)")

    def run(self, a0=0, a1=None):
        """Alg. 2 over simplices [a0, a1)."""
        a1 = len(self.simp) if a1 is None else a1
        r = _load().sv_run(self._h, int(a0), int(a1))
        try:
            return Pieces(r.contents)
        finally:
            _load().sv_free_result(r)

    def run_list(self, simplices):
        """Alg. 2 over the listed simplices (a sample of the mesh)."""
        lst = np.ascontiguousarray(simplices, dtype=np.int64)
        r = _load().sv_run_list(self._h, lst.ctypes.data_as(ctypes.c_void_p), len(lst))
        try:
            return Pieces(r.contents)
        finally:
            _load().sv_free_result(r)

    def close(self):
        if getattr(self, "_h", None):
            _load().sv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
