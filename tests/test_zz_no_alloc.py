"""vd_get_pieces_noalloc: piece export into caller-owned buffers, no device allocation.

Callers whose device memory belongs to a host framework's allocator or arena,
or whose steady-state loop must not trigger a synchronising cudaMalloc, cannot
let the library allocate while they read the pieces.  The no-allocation entry
point must give exactly what vd_get_pieces gives (integer arrays bit for bit,
measures and moments identical), on consecutive calls that share its fixed
scratch array.  Kept in a file of its own, collected after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(d, np_cap, nf_cap):
    lib = B.load()
    simplex = torch.full((np_cap,), -7, dtype=torch.int32, device="cuda")
    site = torch.full((np_cap,), -7, dtype=torch.int32, device="cuda")
    off = torch.full((np_cap + 1,), -7, dtype=torch.int64, device="cuda")
    flags = torch.full((max(nf_cap, 1),), -7, dtype=torch.int32, device="cuda")
    meas = torch.full((np_cap,), -7.0, dtype=d.dtype, device="cuda")
    mom = torch.full((np_cap, 3), -7.0, dtype=d.dtype, device="cuda")
    n_p, n_f = ctypes.c_int64(-1), ctypes.c_int64(-1)
    rc = lib.vd_get_pieces_noalloc(d._h, simplex.data_ptr(), site.data_ptr(), off.data_ptr(), flags.data_ptr(),
                                   meas.data_ptr(), mom.data_ptr(), np_cap, nf_cap, ctypes.byref(n_p),
                                   ctypes.byref(n_f))
    torch.cuda.synchronize()
    return rc, n_p.value, n_f.value, dict(simplex=simplex, site=site, flag_off=off, flags=flags, measure=meas,
                                         moment=mom)


def _check_same(ref, got, np_, nf):
    assert np_ == len(ref["simplex"]) and nf == len(ref["flags"])
    for k in ("simplex", "site"):
        assert torch.equal(got[k][:np_], ref[k]), k
    assert torch.equal(got["flag_off"][:np_ + 1], ref["flag_off"])
    assert torch.equal(got["flags"][:nf], ref["flags"])
    assert torch.equal(got["measure"][:np_], ref["measure"])
    assert torch.equal(got["moment"][:np_], ref["moment"])


def test_noalloc_export_matches_get_pieces(gpu):
    v, s = I.kuhn_lattice_tets(2)
    for n, seed in ((3000, I.SEED_BASE + 71), (6000, I.SEED_BASE + 72)):
        w = dict(mode=4, sites=I.uniform_sites(n, 3, seed), verts=v, simp=s, f64=False)
        d = B.diagram_from_workload(w)
        r = d.compute()
        ref = d.pieces()
        np_ref, nf_ref = len(ref["simplex"]), len(ref["flags"])
        assert np_ref == r["stats"]["pairs"]
        # two calls in a row on the shared scratch, both equal to vd_get_pieces
        for _ in range(2):
            rc, np_, nf, got = _noalloc(d, np_ref + 5, nf_ref + 5)
            assert rc == 0, B.ERRORS.get(rc, rc)
            _check_same(ref, got, np_, nf)
        # capacities below the sizes are rejected
        rc, _, _, _ = _noalloc(d, np_ref - 1, nf_ref + 5)
        assert rc == -4
        rc, _, _, _ = _noalloc(d, np_ref, nf_ref - 1)
        assert rc == -4
        d.close()


def test_noalloc_export_fp64_planar(gpu):
    w = I.workload("square")
    d = B.diagram_from_workload(w)
    d.compute()
    ref = d.pieces()
    for _ in range(2):
        rc, np_, nf, got = _noalloc(d, len(ref["simplex"]), len(ref["flags"]))
        assert rc == 0
        _check_same(ref, got, np_, nf)
    d.close()


def _buffers(np_cap, nf_cap, dtype):
    return dict(simplex=torch.full((np_cap,), -7, dtype=torch.int32, device="cuda"),
                site=torch.full((np_cap,), -7, dtype=torch.int32, device="cuda"),
                flag_off=torch.full((np_cap + 1,), -7, dtype=torch.int64, device="cuda"),
                flags=torch.full((max(nf_cap, 1),), -7, dtype=torch.int32, device="cuda"),
                measure=torch.full((np_cap,), -7.0, dtype=dtype, device="cuda"),
                moment=torch.full((np_cap, 3), -7.0, dtype=dtype, device="cuda"))


def _call_into(d, b, np_cap, nf_cap):
    n_p, n_f = ctypes.c_int64(-1), ctypes.c_int64(-1)
    rc = B.load().vd_get_pieces_noalloc(d._h, b["simplex"].data_ptr(), b["site"].data_ptr(),
                                        b["flag_off"].data_ptr(), b["flags"].data_ptr(), b["measure"].data_ptr(),
                                        b["moment"].data_ptr(), np_cap, nf_cap, ctypes.byref(n_p),
                                        ctypes.byref(n_f))
    return rc, n_p.value, n_f.value


def test_noalloc_on_fresh_context_allocates_nothing(gpu):
    """On a context whose pieces were never exported, two no-allocation calls in a
    row into buffers the caller made beforehand leave the device's free memory as
    it was, and a later vd_get_pieces gives the same pieces."""
    w = I.workload("cube", n=8000)
    d = B.diagram_from_workload(w)
    r = d.compute()
    np_ = int(r["stats"]["pairs"])
    nf_cap = 64 * np_
    bufs = [_buffers(np_, nf_cap, d.dtype) for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out = [_call_into(d, b, np_, nf_cap) for b in bufs]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref = d.pieces()
    for (rc, n_p, n_f), b in zip(out, bufs):
        assert rc == 0, B.ERRORS.get(rc, rc)
        _check_same(ref, b, n_p, n_f)
    d.close()
