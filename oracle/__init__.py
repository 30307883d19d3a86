"""CPU FP64 oracle for clipped / restricted Voronoi pieces (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path (``paper_2509_07175_b300``)
never does; the two share no code.  The arithmetic lives in ``vd_oracle.c``
(see its header for what is computed and which passage of the paper each part
follows: Eq. 1 for the cell, Sec. 2.2 for the face flags).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (brute force, lattice closed form, n=1 and n=2
closed forms, partition invariants, neighbour symmetry; power weights: equal
weights reduce to the Voronoi diagram, the two-site weighted closed form,
brute force against the generalised security radius, a planted sign flip).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_2D, MODE_SURFACE, MODE_3D = 2, 3, 4
FLAG_BOUNDARY = -(2 ** 31)
STAT_NAMES = ("fast", "exact64", "exact128", "tie", "uncertain", "clips", "pieces", "error")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU code involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread", "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [
        ("np", ctypes.c_int64),
        ("a", ctypes.POINTER(ctypes.c_int32)),
        ("i", ctypes.POINTER(ctypes.c_int32)),
        ("meas", ctypes.POINTER(ctypes.c_double)),
        ("m1", ctypes.POINTER(ctypes.c_double)),
        ("foff", ctypes.POINTER(ctypes.c_int64)),
        ("flags", ctypes.POINTER(ctypes.c_int32)),
        ("fmeas", ctypes.POINTER(ctypes.c_double)),
        ("status", ctypes.POINTER(ctypes.c_int32)),
        ("stats", ctypes.c_int64 * 8),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, P,
                                   ctypes.c_int, ctypes.c_int]
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_weights.argtypes = [P, P]
        lib.orc_set_weights.restype = None
        lib.orc_adjacency.argtypes = [P, P]
        lib.orc_adjacency.restype = ctypes.c_int64
        for f in (lib.orc_pieces, lib.orc_enumerate, lib.orc_site_pieces):
            f.restype = ctypes.POINTER(_Result)
        lib.orc_pieces.argtypes = [P, ctypes.c_int64, P, P]
        lib.orc_enumerate.argtypes = [P]
        lib.orc_site_pieces.argtypes = [P, ctypes.c_int64, P]
        lib.orc_free_result.argtypes = [ctypes.POINTER(_Result)]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Pieces:
    """Pieces P_{a,i} with measure, first moment (frame of v_i) and face flags."""

    def __init__(self, res: _Result):
        n = res.np
        self.a = np.ctypeslib.as_array(res.a, (n,)).astype(np.int64) if n else np.zeros(0, np.int64)
        self.i = np.ctypeslib.as_array(res.i, (n,)).astype(np.int64) if n else np.zeros(0, np.int64)
        self.meas = np.ctypeslib.as_array(res.meas, (n,)).copy() if n else np.zeros(0)
        self.m1 = np.ctypeslib.as_array(res.m1, (n, 3)).copy() if n else np.zeros((0, 3))
        self.status = np.ctypeslib.as_array(res.status, (n,)).copy() if n else np.zeros(0, np.int32)
        self.foff = np.ctypeslib.as_array(res.foff, (n + 1,)).copy()
        nf = int(self.foff[-1])
        self.flags = np.ctypeslib.as_array(res.flags, (nf,)).copy() if nf else np.zeros(0, np.int32)
        self.fmeas = np.ctypeslib.as_array(res.fmeas, (nf,)).copy() if nf else np.zeros(0)
        self.stats = dict(zip(STAT_NAMES, list(res.stats)))

    def __len__(self):
        return len(self.a)

    def face_flags(self, p):
        return self.flags[self.foff[p]:self.foff[p + 1]]

    def face_measures(self, p):
        return self.fmeas[self.foff[p]:self.foff[p + 1]]

    def nonempty(self):
        return self.meas > 0

    def topology(self):
        """{(a, i): sorted tuple of face flags} over pieces of positive measure."""
        out = {}
        for p in np.nonzero(self.meas > 0)[0]:
            out[(int(self.a[p]), int(self.i[p]))] = tuple(sorted(int(f) for f in self.face_flags(p)))
        return out


class Oracle:
    """Context over one input (sites, mesh).

    ``mode``: 2 (2D, sites and triangles in z=0), 3 (surface triangles in R^3),
    4 (tetrahedra).  ``brute``: clip by all n-1 bisectors (tiny inputs only).
    """

    def __init__(self, mode, sites, verts, simp, brute=False, nthreads=None, weights=None):
        self.mode = int(mode)
        self.sites = np.ascontiguousarray(sites, dtype=np.float64).reshape(-1, 3)
        self.verts = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3)
        self.simp = np.ascontiguousarray(simp, dtype=np.int32)
        self.k = self.simp.shape[1]
        assert (self.mode == MODE_3D) == (self.k == 4)
        nt = nthreads or os.cpu_count() or 1
        self.nthreads = nt
        lib = _load()
        self._h = lib.orc_create(self.mode, len(self.sites), _ptr(self.sites), len(self.verts), _ptr(self.verts),
                                 len(self.simp), _ptr(self.simp), int(bool(brute)), int(nt))
        if weights is not None:
            # power diagram: |x - v_i|^2 - w_i <= |x - v_j|^2 - w_j
            self.weights = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
            assert len(self.weights) == len(self.sites)
            lib.orc_set_weights(self._h, _ptr(self.weights))

    def close(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def adjacency(self):
        out = np.empty((len(self.simp), self.k), dtype=np.int32)
        _load().orc_adjacency(self._h, _ptr(out))
        return out

    def _wrap(self, r):
        try:
            return Pieces(r.contents)
        finally:
            _load().orc_free_result(r)

    def pieces(self, a, i):
        a = np.ascontiguousarray(a, dtype=np.int64)
        i = np.ascontiguousarray(i, dtype=np.int64)
        return self._wrap(_load().orc_pieces(self._h, len(a), _ptr(a), _ptr(i)))

    def enumerate(self):
        return self._wrap(_load().orc_enumerate(self._h))

    def all_sites(self):
        """Every non-empty piece of every site: the per-site form over all sites
        (parallel over sites; the same pieces as enumerate(), which works simplex
        by simplex -- see tests/test_oracle_pins.py)"""
        return self.site_pieces(np.arange(len(self.sites)))

    def site_pieces(self, sites):
        s = np.ascontiguousarray(sites, dtype=np.int64)
        return self._wrap(_load().orc_site_pieces(self._h, len(s), _ptr(s)))


def per_site(n, sites, pieces: Pieces, site_ids=None):
    """Per-site measure, centroid (global frame) and sorted neighbour lists.

    measure_i = sum_a |P_{a,i}|; centroid_i = v_i + sum_a M1_{a,i} / measure_i
    (v_i for an empty cell); neighbours = bisector flags of faces of positive
    measure over the site's pieces.
    """
    ids = np.arange(n) if site_ids is None else np.asarray(site_ids)
    meas = np.zeros(n)
    m1 = np.zeros((n, 3))
    np.add.at(meas, pieces.i, pieces.meas)
    np.add.at(m1, pieces.i, pieces.m1)
    cen = sites[:n].copy()
    ok = meas > 0
    cen[ok] += m1[ok] / meas[ok, None]
    nbrs = [set() for _ in range(n)]
    for p in range(len(pieces)):
        if pieces.meas[p] <= 0:
            continue
        for f in pieces.face_flags(p):
            if f >= 0:
                nbrs[pieces.i[p]].add(int(f))
    return meas[ids], cen[ids], [sorted(nbrs[i]) for i in ids]
