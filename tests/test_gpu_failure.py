"""Bounded failure paths: each fixed capacity and each bounded loop or wait of the
library returns its error code, a corrupted mesh is rejected by validation, and
the same context then computes the diagram correctly again.

Every failure is made on the host: options that shrink a capacity or a limit, or a
mesh corrupted before it is passed in.  Nothing here faults, traps or hangs the
GPU: every capacity check in the kernels runs before the write it guards (queue
slot, pair-set probe, flag range, polytope slot), every wait of an idle worker is
bounded by wall time, and the kernels that read the flood's per-slot outputs
return at once once the status is set.
"""
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_full

pytestmark = pytest.mark.gpu

ERR_CAPACITY, ERR_LIMIT, ERR_DOMAIN, ERR_STATE = -4, -5, -6, -8


def _cube_case(n=600, seed=I.SEED_BASE + 0x300):
    v, s = I.kuhn_lattice_tets(2)
    return dict(name="fail", mode=B.MODE_3D, sites=I.uniform_sites(n, 3, seed), verts=v, simp=s, f64=False)


_ORACLE = {}


def _oracle(w):
    key = (w["name"], len(w["sites"]), w["mode"])
    if key not in _ORACLE:
        _ORACLE[key] = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"]).enumerate()
    return _ORACLE[key]


def _tensors(w):
    dim = 2 if w["mode"] == B.MODE_2D else 3
    v = torch.tensor(w["verts"][:, :dim], dtype=torch.float32, device="cuda")
    t = torch.tensor(w["simp"], dtype=torch.int32, device="cuda")
    return v, t


def _recovers(d, w, reset_domain=False):
    """Default options (and the domain set again when its buffers were sized by the
    failing options): the next compute on the same context matches the oracle."""
    d.set_options()
    if reset_domain:
        d.set_domain(*_tensors(w))
    r = d.compute()
    assert r["status"] == 0
    compare_full(w, r, d.pieces(), _oracle(w))


def _failed_compute(d, code):
    r = d.compute(check=False)
    assert r["status"] == code, (r["status"], code)
    # the pieces of a failed compute are incomplete: the export refuses them
    with pytest.raises(B.VDError) as e:
        d.pieces()
    assert e.value.code == ERR_STATE


def test_queue_capacity(gpu):
    """A work queue too small for the pairs: VD_ERR_CAPACITY (the slot index is
    checked before the queue write), then the context recovers."""
    w = _cube_case()
    d = B.diagram_from_workload(w, options=dict(queue_capacity=64))
    _failed_compute(d, ERR_CAPACITY)
    _recovers(d, w, reset_domain=True)
    d.close()


def test_queue_capacity_box_form(gpu):
    """The box form seeds one pair per site straight into the queue: a queue
    smaller than the site count is refused per slot, not overrun."""
    w = I.workload("box", n=3000)
    d = B.diagram_from_workload(w, options=dict(queue_capacity=1000))
    r = d.compute(check=False)
    assert r["status"] == ERR_CAPACITY
    d.set_options()
    d.set_box(*w["box"])
    r = d.compute()
    assert r["status"] == 0
    m = r["measure"].double().cpu().numpy()
    assert abs(m.sum() - 1.0) <= 1e-5
    d.close()


def test_max_clips(gpu):
    """One clip per pair allowed: the bounded clip loop stops with VD_ERR_LIMIT."""
    w = _cube_case()
    d = B.diagram_from_workload(w, options=dict(max_clips=1))
    _failed_compute(d, ERR_LIMIT)
    _recovers(d, w)
    d.close()


def test_search_limits_degrade_to_witness(gpu):
    """Plain search with one start-point step and one search step: a search that
    runs out clips by the corner's certified closer site instead (a valid
    bisector, Omega_i lies in its half-space), so the diagram is unchanged and
    only the fallback count grows."""
    w = _cube_case()
    d = B.diagram_from_workload(w, options=dict(max_search=1, max_lambda=1, stats=1))
    r = d.compute()
    assert r["status"] == 0 and r["stats"]["fallback"] > 0
    compare_full(w, r, d.pieces(), _oracle(w))
    d.close()


def test_wait_limit(gpu):
    """Idle workers may wait one nanosecond for a queue slot: the first worker that
    finds no pair while others still work gives up with VD_ERR_LIMIT (the wait is
    bounded by the global timer, so nothing spins unboundedly)."""
    w = _cube_case()
    d = B.diagram_from_workload(w, options=dict(wait_limit_s=1e-9))
    _failed_compute(d, ERR_LIMIT)
    _recovers(d, w)
    d.close()


def test_error_then_lloyd_graph_recovers(gpu):
    """A failing limit inside a captured Lloyd graph is reported once at the end
    and leaves the sites as they were (no update from an unfinished diagram); the
    same context then relaxes normally."""
    w = _cube_case(n=300, seed=I.SEED_BASE + 0x301)
    d = B.diagram_from_workload(w, options=dict(max_clips=1))
    before = d.sites().cpu()
    with pytest.raises(B.VDError) as e:
        d.lloyd(3, use_graph=True)
    assert e.value.code == ERR_LIMIT
    assert torch.equal(d.sites().cpu(), before)
    d.set_options()
    d.lloyd(3, use_graph=True)
    r = d.compute()
    assert r["status"] == 0
    m = r["measure"].double().cpu().numpy()
    assert abs(m.sum() - 1.0) <= 1e-5
    assert not torch.equal(d.sites().cpu(), before)
    d.close()


@pytest.mark.parametrize("kind", ["index_high", "index_negative", "zero_volume", "face_three_tets"])
def test_corrupted_tet_mesh(gpu, kind):
    """Mesh validation: an index out of range, a tetrahedron of zero volume and a
    face shared by three tetrahedra are rejected with VD_ERR_DOMAIN; setting the
    valid mesh again restores a correct compute."""
    w = _cube_case()
    d = B.diagram_from_workload(w)
    v, t = _tensors(w)
    bad = t.clone()
    if kind == "index_high":
        bad[3, 2] = v.shape[0]
    elif kind == "index_negative":
        bad[5, 0] = -1
    elif kind == "zero_volume":
        bad[7, 3] = bad[7, 0]
    else:  # a copy of tet 0: its interior faces are now shared by three tets
        bad = torch.cat([t, t[:1]], 0)
    assert d.set_domain(v, bad, check=False) == ERR_DOMAIN
    # the failed call dropped the old domain: computing now is out of order
    assert d.compute(check=False)["status"] == ERR_STATE
    d.set_domain(v, t)
    r = d.compute()
    assert r["status"] == 0
    compare_full(w, r, d.pieces(), _oracle(w))
    d.close()


@pytest.mark.parametrize("kind", ["zero_area", "edge_three_tris"])
def test_corrupted_surface_mesh(gpu, kind):
    """The same validation on a triangle mesh in 3D (restricted diagram)."""
    v, s = I.torus_domain(nu=40, nv=12)
    sites = I.surface_sites(400, v, s, I.SEED_BASE + 0x302)
    w = dict(name="failsurf", mode=B.MODE_SURFACE, sites=sites, verts=v, simp=s, f64=False)
    d = B.diagram_from_workload(w)
    vt, tt = _tensors(w)
    if kind == "zero_area":
        bad = tt.clone()
        bad[2, 1] = bad[2, 0]
    else:
        bad = torch.cat([tt, tt[:1]], 0)
    assert d.set_domain(vt, bad, check=False) == ERR_DOMAIN
    d.set_domain(vt, tt)
    r = d.compute()
    assert r["status"] == 0
    compare_full(w, r, d.pieces(), _oracle(w))
    d.close()


@pytest.mark.parametrize("name,n,opts", [
    ("fail", 600, dict(mapping=1)),                      # warp per pair, 3D
    ("fail", 600, dict(mapping=2)),                      # thread per pair, 3D
    ("fail", 600, dict(learned=1, topk=16, split=1)),    # learned form with the split
    ("torus", 3000, dict(mapping=1)),                    # polygon form, surface
])
def test_forced_float64_path(gpu, name, n, opts):
    """A filter failure forced from the host (vd_options.force_exact): every clip
    decision and every new corner takes the float64 path.  The diagram matches
    the oracle with the same bar, the neighbours equal the filtered run's, and
    the float64 count covers the clip decisions."""
    if name == "fail":
        w = _cube_case(n)
    else:  # a small torus (1,600 triangles), sites on it
        v, s = I.torus_domain(nu=40, nv=20)
        w = dict(name="torus_small", mode=B.MODE_SURFACE, sites=I.surface_sites(n, v, s, I.SEED_BASE + 0x330),
                 verts=v, simp=s, f64=False)
    d = B.diagram_from_workload(w, options=dict(opts, stats=1))
    ref = d.compute()
    d.set_options(**dict(opts, stats=1, force_exact=1))
    r = d.compute()
    assert r["status"] == 0 and r["stats"]["uncertain"] == 0
    assert r["stats"]["fp64"] > 3 * ref["stats"]["fp64"]
    assert torch.equal(r["nbr_off"], ref["nbr_off"]) and torch.equal(r["nbr_idx"], ref["nbr_idx"])
    compare_full(w, r, d.pieces(), _oracle(w), split=bool(opts.get("split")))
    d.close()
