"""ctypes binding of libvd (include/vd.h): argument marshalling only.

Every step of the computation runs in libvd's CUDA kernels; torch supplies the
device memory (``tensor.data_ptr()``) and the stream.  Loading fails loudly if
the library is missing or no CUDA device is present -- there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvd.so")

VD_F32, VD_F64 = 0, 1
MODE_2D, MODE_SURFACE, MODE_3D = 2, 3, 4
FLAG_BOUNDARY = -(2 ** 31)
PROPOSAL_DISTANCE, PROPOSAL_MLP = 0, 1
MLP_NPARAM, MLP_NIN, MLP_NOUT = 12448, 96, 32
STAT_NAMES = ("pairs", "nonempty", "nn_queries", "corner_tests", "clips", "lambda_steps", "search_steps",
              "fp64", "uncertain", "ties", "sites_scanned", "learned_hits", "fallback", "launches", "illcond")
PHASE_NAMES = ("grid", "delta", "seed", "clip", "reduce")

ERRORS = {0: "ok", -1: "VD_ERR_ARG", -2: "VD_ERR_CUDA", -3: "VD_ERR_OOM", -4: "VD_ERR_CAPACITY",
          -5: "VD_ERR_LIMIT", -6: "VD_ERR_DOMAIN", -7: "VD_ERR_UNCERTAIN", -8: "VD_ERR_STATE",
          -9: "VD_ERR_DUPLICATE", -10: "VD_ERR_IO"}


class VDError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({code})")


class Options(ctypes.Structure):
    _fields_ = [("learned", ctypes.c_int), ("mapping", ctypes.c_int), ("chunk", ctypes.c_int),
                ("stats", ctypes.c_int), ("queue_capacity", ctypes.c_int64), ("max_clips", ctypes.c_int),
                ("max_search", ctypes.c_int), ("max_lambda", ctypes.c_int), ("wait_limit_s", ctypes.c_double),
                ("timing", ctypes.c_int), ("grid_density", ctypes.c_double), ("topk", ctypes.c_int),
                ("proposal", ctypes.c_int), ("split", ctypes.c_int),
                ("nearest", ctypes.c_int), ("force_exact", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_pieces", ctypes.c_int64),
                ("dtype", ctypes.c_int), ("measure", ctypes.c_void_p), ("centroid", ctypes.c_void_p),
                ("nbr_off", ctypes.c_void_p), ("nbr_idx", ctypes.c_void_p), ("stats", ctypes.c_int64 * 32),
                ("status", ctypes.c_int), ("phase_ms", ctypes.c_double * 8)]


class PiecesC(ctypes.Structure):
    _fields_ = [("n_pieces", ctypes.c_int64), ("simplex", ctypes.c_void_p), ("site", ctypes.c_void_p),
                ("measure", ctypes.c_void_p), ("moment", ctypes.c_void_p), ("flag_off", ctypes.c_void_p),
                ("flags", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libvd.so (raises if absent: the product path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libvd.so not built ({path}); run paper_2509_07175_b300/build.py")
    lib = ctypes.CDLL(path)
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "vd_create": ([ctypes.POINTER(P), P, I64, I, I], I),
        "vd_set_domain": ([P, P, I64, P, I64, I], I),
        "vd_set_options": ([P, ctypes.POINTER(Options)], I),
        "vd_set_stream": ([P, P], I),
        "vd_update_sites": ([P, P], I),
        "vd_update_sites_host": ([P, P], I),
        "vd_compute": ([P, ctypes.POINTER(Result)], I),
        "vd_compute_async": ([P], I),
        "vd_get_status": ([P, ctypes.POINTER(I)], I),
        "vd_get_result": ([P, ctypes.POINTER(Result)], I),
        "vd_model_save": ([P, ctypes.c_char_p], I),
        "vd_model_load": ([P, ctypes.c_char_p], I),
        "vd_copy_result_host": ([P, P, P, P, P], I),
        "vd_lloyd": ([P, I, I], I),
        "vd_get_sites": ([P, P], I),
        "vd_get_pieces": ([P, ctypes.POINTER(PiecesC)], I),
        "vd_set_candidates": ([P, P, I], I),
        "vd_get_pieces_noalloc": ([P, P, P, P, P, P, P, I64, I64, ctypes.POINTER(I64), ctypes.POINTER(I64)], I),
        "vd_mlp_init": ([P, ctypes.c_uint64], I),
        "vd_mlp_set_state": ([P, P, P, P, I64], I),
        "vd_mlp_get_state": ([P, P, P, P, ctypes.POINTER(I64)], I),
        "vd_mlp_features": ([P, P, P], I),
        "vd_mlp_grad": ([P, P, P, I64, P, P], I),
        "vd_mlp_forward": ([P, P, I64, P], I),
        "vd_mlp_train": ([P, P, P, I64, I, I, ctypes.c_float, ctypes.c_uint64, P], I),
        "vd_get_candidate_masks": ([P, P], I),
        "vd_autotune": ([P, ctypes.POINTER(I), ctypes.POINTER(I), P], I),
        "vd_set_box": ([P, P, P], I),
        "vd_create_power2d": ([ctypes.POINTER(P), P, P, I64], I),
        "vd_set_weights": ([P, P], I),
        "vd_set_partition": ([P, P, I], I),
        "vd_get_outbox": ([P, ctypes.POINTER(P), ctypes.POINTER(I64)], I),
        "vd_resume": ([P, P, I64, ctypes.POINTER(I64), ctypes.POINTER(Result)], I),
        "vd_lloyd_step": ([P], I),
        "vd_destroy": ([P], None),
        "vd_strerror": ([I], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return ["vd_create", "vd_set_domain", "vd_set_options", "vd_set_stream", "vd_update_sites",
            "vd_update_sites_host", "vd_compute", "vd_copy_result_host", "vd_lloyd", "vd_get_sites",
            "vd_get_pieces", "vd_set_candidates", "vd_destroy", "vd_strerror", "vd_get_pieces_noalloc",
            "vd_mlp_init", "vd_mlp_set_state", "vd_mlp_get_state", "vd_mlp_features", "vd_mlp_grad",
            "vd_mlp_forward", "vd_mlp_train", "vd_get_candidate_masks", "vd_autotune", "vd_set_box",
            "vd_create_power2d", "vd_compute_async", "vd_get_status", "vd_get_result", "vd_model_save",
            "vd_model_load", "vd_set_weights", "vd_set_partition", "vd_get_outbox", "vd_resume",
            "vd_lloyd_step"]


class _DevArray:
    """Borrowed device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


def _view(ptr, shape, dtype):
    typestr = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4", torch.int64: "<i8"}[dtype]
    n = 1
    for s in shape:
        n *= s
    if n == 0 or not ptr:
        return torch.zeros(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


def _check(code, where):
    if code != 0:
        raise VDError(code, where)


class Diagram:
    """One site set and one simplicial domain on the current CUDA device.

    sites: (n, dim) float32 or float64 CUDA tensor (dim 2 or 3).
    verts: (nv, dim) CUDA tensor of the same dtype; simplices: (m, 3|4) int32.
    """

    def __init__(self, sites, verts=None, simplices=None, options: dict | None = None, stream=None, box=None,
                 weights=None):
        """box = (lo, hi): the axis-aligned box domain (vd_set_box) instead of a mesh.
        weights (n,) with planar sites (n, 2) and a planar triangle mesh: the power
        diagram (vd_create_power2d; the mesh is placed at z = 0)."""
        lib = load()
        if not sites.is_cuda or (box is None and not (verts.is_cuda and simplices.is_cuda)):
            raise ValueError("inputs must be CUDA tensors")
        self._keep = []
        h = ctypes.c_void_p()
        if weights is not None:
            xy = sites.to(torch.float32).contiguous()
            wt = weights.to(device=sites.device, dtype=torch.float32).contiguous()
            _check(lib.vd_create_power2d(ctypes.byref(h), xy.data_ptr(), wt.data_ptr(), xy.shape[0]),
                   "vd_create_power2d")
            self.dtype = torch.float32
            self.n, self.dim = xy.shape[0], 3
            verts = torch.cat([verts.to(torch.float32), torch.zeros((verts.shape[0], 1), dtype=torch.float32,
                                                                    device=verts.device)], 1)
        else:
            self.dtype = sites.dtype
            self.n, self.dim = sites.shape
            s = sites.contiguous()
            _check(lib.vd_create(ctypes.byref(h), s.data_ptr(), self.n, self.dim,
                                 VD_F64 if self.dtype == torch.float64 else VD_F32), "vd_create")
        self._h = h
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        _check(lib.vd_set_stream(h, ctypes.c_void_p(st.cuda_stream)), "vd_set_stream")
        if options:
            self.set_options(**options)
        if box is not None:
            self.set_box(*box)
        else:
            self.set_domain(verts, simplices)
        self.result = None

    def set_box(self, lo, hi):
        """vd_set_box: the axis-aligned box [lo, hi] as a convex domain."""
        lo = (ctypes.c_double * 3)(*[float(x) for x in lo])
        hi = (ctypes.c_double * 3)(*[float(x) for x in hi])
        _check(load().vd_set_box(self._h, lo, hi), "vd_set_box")
        self.m, self.k = 1, 0

    def set_domain(self, verts, simplices, check=True):
        """vd_set_domain with a new mesh; returns the code when check is False."""
        v = verts.to(self.dtype).contiguous()
        t = simplices.to(torch.int32).contiguous()
        code = load().vd_set_domain(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], t.shape[1])
        if check:
            _check(code, "vd_set_domain")
        if code == 0:
            self.m, self.k = t.shape
        return code

    def set_options(self, **kw):
        o = Options()
        for k, v in kw.items():
            setattr(o, k, v)
        _check(load().vd_set_options(self._h, ctypes.byref(o)), "vd_set_options")

    def set_weights(self, weights):
        """Power diagram (3D or surface): site weights (n,) float32, None for the Voronoi diagram."""
        if weights is None:
            _check(load().vd_set_weights(self._h, None), "vd_set_weights")
            return
        wt = weights.to(device="cuda", dtype=torch.float32).contiguous()
        _check(load().vd_set_weights(self._h, wt.data_ptr()), "vd_set_weights")

    def update_sites(self, sites):
        s = sites.to(self.dtype).contiguous()
        _check(load().vd_update_sites(self._h, s.data_ptr()), "vd_update_sites")

    def update_sites_host(self, sites_host):
        _check(load().vd_update_sites_host(self._h, sites_host.data_ptr()), "vd_update_sites_host")

    def compute(self, check=True):
        """Run the diagram; returns dict of torch tensors (copies) and stats."""
        r = Result()
        code = load().vd_compute(self._h, ctypes.byref(r))
        if check:
            _check(code, "vd_compute")
        self.result = r
        return self._pack(r, code)

    def compute_raw(self):
        """vd_compute with no copies (for timing); returns the status code."""
        r = Result()
        return load().vd_compute(self._h, ctypes.byref(r)), r

    def compute_async(self):
        """Enqueue a compute on the diagram's stream (no host synchronisation)."""
        _check(load().vd_compute_async(self._h), "vd_compute_async")

    def status(self):
        """Wait for the stream and read the device status of the last enqueued compute."""
        st = ctypes.c_int()
        _check(load().vd_get_status(self._h, ctypes.byref(st)), "vd_get_status")
        return st.value

    def get_result(self, check=True):
        """The result (copies) of the computation whose status was read last."""
        r = Result()
        _check(load().vd_get_result(self._h, ctypes.byref(r)), "vd_get_result")
        if check:
            _check(int(r.status), "device status")
        self.result = r
        return self._pack(r, int(r.status))

    def set_partition(self, owner, rank):
        """Own the sites with owner[i] == rank (owner: int32 tensor [n]); None: own all."""
        if owner is None:
            _check(load().vd_set_partition(self._h, None, 0), "vd_set_partition")
            return
        o = owner.to(device="cuda", dtype=torch.int32).contiguous()
        _check(load().vd_set_partition(self._h, o.data_ptr(), int(rank)), "vd_set_partition")

    def outbox(self):
        """Pairs found for other ranks' sites (int64 keys (simplex << 32) | site, a copy)."""
        k, cnt = ctypes.c_void_p(), ctypes.c_int64()
        _check(load().vd_get_outbox(self._h, ctypes.byref(k), ctypes.byref(cnt)), "vd_get_outbox")
        n = int(cnt.value)
        if n == 0:
            return torch.zeros(0, dtype=torch.int64, device="cuda")
        return _view(k.value, (n,), torch.int64).clone()

    def resume(self, keys, check=True):
        """Continue the computation with received pairs; returns (result, new pairs)."""
        kk = keys.to(device="cuda", dtype=torch.int64).contiguous()
        r, added = Result(), ctypes.c_int64()
        code = load().vd_resume(self._h, kk.data_ptr() if kk.numel() else None, int(kk.numel()),
                                ctypes.byref(added), ctypes.byref(r))
        if check:
            _check(code, "vd_resume")
        self.result = r
        return self._pack(r, code), int(added.value)

    def lloyd_step(self):
        """Move every site with a non-empty cell to its centroid (the last computation's)."""
        _check(load().vd_lloyd_step(self._h), "vd_lloyd_step")

    def model_save(self, path):
        _check(load().vd_model_save(self._h, os.fsencode(path)), "vd_model_save")

    def model_load(self, path):
        _check(load().vd_model_load(self._h, os.fsencode(path)), "vd_model_load")

    def _pack(self, r, code):
        n = int(r.n)
        out = {
            "status": code,
            "measure": _view(r.measure, (n,), self.dtype).clone(),
            "centroid": _view(r.centroid, (n, 3), self.dtype).clone(),
            "nbr_off": _view(r.nbr_off, (n + 1,), torch.int64).clone(),
            "nbr_idx": _view(r.nbr_idx, (int(r.nnz),), torch.int32).clone(),
            "n_pieces": int(r.n_pieces),
            "stats": dict(zip(STAT_NAMES, [int(x) for x in r.stats][:len(STAT_NAMES)]),
                          error_line=int(r.stats[15]), diag=[int(x) for x in r.stats[16:24]],
                          list_tests=int(r.stats[30]), whole_cells=int(r.stats[24]),
                          boundary_sites=int(r.stats[25]), bisector_faces=int(r.stats[26]),
                          excess_clips=int(r.stats[27]), mapping=int(r.stats[31]) & 255,
                          chunk=(int(r.stats[31]) >> 8) & 255, nearest=int(r.stats[31]) >> 16),
            "phase_ms": dict(zip(PHASE_NAMES, [float(x) for x in r.phase_ms][:len(PHASE_NAMES)])),
        }
        return out

    def copy_result_host(self, measure, centroid, nbr_off=None, nbr_idx=None):
        f = lambda t: None if t is None else t.data_ptr()  # noqa: E731
        _check(load().vd_copy_result_host(self._h, f(measure), f(centroid), f(nbr_off), f(nbr_idx)),
               "vd_copy_result_host")

    def pieces(self):
        p = PiecesC()
        _check(load().vd_get_pieces(self._h, ctypes.byref(p)), "vd_get_pieces")
        np_ = int(p.n_pieces)
        off = _view(p.flag_off, (np_ + 1,), torch.int64).clone()
        nf = int(off[-1].item()) if np_ else 0
        return {
            "simplex": _view(p.simplex, (np_,), torch.int32).clone(),
            "site": _view(p.site, (np_,), torch.int32).clone(),
            "measure": _view(p.measure, (np_,), self.dtype).clone(),
            "moment": _view(p.moment, (np_, 3), self.dtype).clone(),
            "flag_off": off,
            "flags": _view(p.flags, (nf,), torch.int32).clone(),
        }

    def lloyd(self, iters, use_graph=True):
        _check(load().vd_lloyd(self._h, int(iters), int(bool(use_graph))), "vd_lloyd")

    def sites(self):
        out = torch.empty((self.n, 3), dtype=self.dtype, device="cuda")
        _check(load().vd_get_sites(self._h, out.data_ptr()), "vd_get_sites")
        torch.cuda.synchronize()
        return out

    def set_candidates(self, cand):
        if cand is None:
            _check(load().vd_set_candidates(self._h, None, 0), "vd_set_candidates")
            return
        c = cand.to(torch.int32).contiguous()
        self._keep.append(c)
        _check(load().vd_set_candidates(self._h, c.data_ptr(), c.shape[1]), "vd_set_candidates")

    # ----- learned proposal network (vd_mlp_*) -----
    def mlp_init(self, seed):
        _check(load().vd_mlp_init(self._h, int(seed)), "vd_mlp_init")

    def mlp_set_state(self, params, adam_m=None, adam_v=None, step=0):
        ts = [None if t is None else t.to(device="cuda", dtype=torch.float32).contiguous()
              for t in (params, adam_m, adam_v)]
        f = lambda t: None if t is None else t.data_ptr()  # noqa: E731
        _check(load().vd_mlp_set_state(self._h, f(ts[0]), f(ts[1]), f(ts[2]), int(step)), "vd_mlp_set_state")
        torch.cuda.current_stream().synchronize()

    def mlp_get_state(self):
        p, m, v = (torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda") for _ in range(3))
        step = ctypes.c_int64()
        _check(load().vd_mlp_get_state(self._h, p.data_ptr(), m.data_ptr(), v.data_ptr(), ctypes.byref(step)),
               "vd_mlp_get_state")
        return {"params": p, "adam_m": m, "adam_v": v, "step": int(step.value)}

    def mlp_features(self, features=True, labels=True):
        """Network inputs (bf16 [n, 96]) and neighbour labels (int32 bit masks [n]) of the last compute."""
        x = torch.empty((self.n, MLP_NIN), dtype=torch.bfloat16, device="cuda") if features else None
        y = torch.empty(self.n, dtype=torch.int32, device="cuda") if labels else None
        _check(load().vd_mlp_features(self._h, None if x is None else x.data_ptr(),
                                      None if y is None else y.data_ptr()), "vd_mlp_features")
        return x, y

    def mlp_grad(self, x, y):
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(load().vd_mlp_grad(self._h, x.data_ptr(), y.data_ptr(), x.shape[0], g.data_ptr(), loss.data_ptr()),
               "vd_mlp_grad")
        return g, loss

    def mlp_forward(self, x):
        z = torch.empty((x.shape[0], MLP_NOUT), dtype=torch.float32, device="cuda")
        _check(load().vd_mlp_forward(self._h, x.data_ptr(), x.shape[0], z.data_ptr()), "vd_mlp_forward")
        return z

    def autotune(self):
        """Time every clip-kernel mapping on the current sites; returns the choice and the times."""
        m, ch = ctypes.c_int(), ctypes.c_int()
        times = (ctypes.c_float * 12)()
        _check(load().vd_autotune(self._h, ctypes.byref(m), ctypes.byref(ch), times), "vd_autotune")
        names = tuple(f"{mp},{k}" for mp in ("warp", "thread") for k in (1, 2, 4, 8, 16)) + ("list32", "list64")
        return {"mapping": m.value, "chunk": ch.value,
                "times_ms": {nm: float(t) for nm, t in zip(names, times) if t >= 0}}

    def candidate_masks(self):
        """Candidate bit masks (int32 [n]) of the last learned-form compute."""
        m = torch.empty(self.n, dtype=torch.int32, device="cuda")
        _check(load().vd_get_candidate_masks(self._h, m.data_ptr()), "vd_get_candidate_masks")
        return m

    def mlp_train(self, x, y, batch=4096, epochs=3, lr=1e-3, seed=0):
        losses = (ctypes.c_float * int(epochs))()
        _check(load().vd_mlp_train(self._h, x.data_ptr(), y.data_ptr(), x.shape[0], int(batch), int(epochs),
                                   float(lr), int(seed), losses), "vd_mlp_train")
        return [float(v) for v in losses]

    def close(self):
        if getattr(self, "_h", None):
            load().vd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def diagram_from_workload(w: dict, device="cuda", options=None):
    """Build a Diagram from an ``inputs.workload`` dict."""
    dt = torch.float64 if w["f64"] else torch.float32
    dim = 2 if w["mode"] == MODE_2D else 3
    s = torch.tensor(w["sites"][:, :dim], dtype=dt, device=device)
    if w.get("box") is not None:
        return Diagram(s, options=options, box=w["box"])
    v = torch.tensor(w["verts"][:, :dim], dtype=dt, device=device)
    t = torch.tensor(w["simp"], dtype=torch.int32, device=device)
    return Diagram(s, v, t, options=options)
