"""Batching: the clip kernel's mappings (one warp or one thread per pair) and
queue chunks, and the autotuner that picks among them.  Every mapping computes
the same diagram bit for bit (exact sign decisions; canonical integration with
one summation order), so the autotuner's choice never changes the output."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_full

pytestmark = pytest.mark.gpu

KEYS = ("measure", "centroid", "nbr_off", "nbr_idx")
MAPS = [(1, 1), (1, 4), (2, 1), (2, 4), (2, 16)]


def _same(a, b, tag):
    for k in KEYS:
        assert torch.equal(a[k], b[k]), (tag, k)


def _topology(d):
    p = d.pieces()
    m = p["measure"].double().cpu().numpy()
    a = p["simplex"].cpu().numpy()
    i = p["site"].cpu().numpy()
    off = p["flag_off"].cpu().numpy()
    fl = p["flags"].cpu().numpy()
    out = {}
    for q in np.nonzero(m > 0)[0]:
        out[(int(a[q]), int(i[q]))] = (m[q], tuple(sorted(int(x) for x in fl[off[q]:off[q + 1]])))
    return out


@pytest.mark.parametrize("name,n", [("cube", 20000), ("shell", 30000), ("cube", 3000)])
@pytest.mark.parametrize("form", ["plain", "learned"])
def test_mappings_bit_identical(gpu, name, n, form):
    w = I.workload(name, n=n)
    d = B.diagram_from_workload(w)
    extra = dict(learned=1, topk=16) if form == "learned" else {}
    ref, ref_top = None, None
    for m, ch in MAPS:
        d.set_options(mapping=m, chunk=ch, stats=1, **extra)
        r = d.compute()
        assert r["status"] == 0 and r["stats"]["uncertain"] == 0
        assert r["stats"]["mapping"] == m and r["stats"]["chunk"] == ch
        top = _topology(d)
        if ref is None:
            ref, ref_top = r, top
            continue
        _same(ref, r, (m, ch))
        assert top == ref_top, (m, ch)   # pieces: same pairs, bit-equal measures, same flags
    d.close()


def test_thread_mapping_against_oracle(gpu):
    """The thread-per-pair form on its own against the oracle (cube, 2,000 sites,
    6 tets and a 2x2x2 Kuhn lattice of 48 tets)."""
    for verts, simp in (I.cube_6tet(), I.kuhn_lattice_tets(2)):
        sites = I.uniform_sites(2000, 3, I.SEED_BASE + 0x140)
        w = dict(name="cube", mode=4, sites=sites, verts=verts, simp=simp, f64=False)
        d = B.diagram_from_workload(w, options=dict(mapping=2, chunk=1))
        r = d.compute()
        assert r["status"] == 0
        p = d.pieces()
        op = O.Oracle(4, sites, verts, simp).enumerate()
        compare_full(w, r, p, op)
        d.close()


def test_network_ranking_with_thread_mapping(gpu):
    w = I.workload("shell", n=30000)
    d = B.diagram_from_workload(w)
    d.set_options(mapping=1)
    plain = d.compute()
    d.mlp_init(5)
    d.set_options(mapping=2, chunk=4, learned=1, proposal=B.PROPOSAL_MLP, topk=8)
    _same(plain, d.compute(), "thread+network")
    d.close()


def test_autotune_choice_and_cache(gpu):
    w = I.workload("cube", n=50000)
    d = B.diagram_from_workload(w)
    d.set_options(mapping=1)
    ref = d.compute()
    d.set_options(mapping=0, stats=1)
    t = d.autotune()
    # every warp chunk and thread chunk 1 are timed; the other thread chunks only
    # when thread chunk 1 beat the best warp chunk
    tm = t["times_ms"]
    warp = {f"warp,{k}" for k in (1, 2, 4, 8, 16)}
    thread = {f"thread,{k}" for k in (1, 2, 4, 8, 16)}
    assert warp | {"thread,1"} <= set(tm) <= warp | thread
    if tm["thread,1"] >= min(tm[k] for k in warp):
        assert set(tm) == warp | {"thread,1"}
    else:
        assert set(tm) == warp | thread
    assert all(v > 0 for v in tm.values())
    best = min(t["times_ms"], key=t["times_ms"].get)
    assert best == f"{'warp' if t['mapping'] == 1 else 'thread'},{t['chunk']}"
    r = d.compute()   # uses the cached choice
    assert (r["stats"]["mapping"], r["stats"]["chunk"]) == (t["mapping"], t["chunk"])
    _same(ref, r, "autotuned")
    print("autotune cube 50k:", t)
    d.close()


def test_polygon_modes_fall_back_to_warp(gpu):
    for name, n in (("square", 1000), ("torus", 20000)):
        w = I.workload(name, n=n)
        d = B.diagram_from_workload(w)
        d.set_options(mapping=1)
        ref = d.compute()
        d.set_options(mapping=2, chunk=4, stats=1)
        r = d.compute()
        assert r["stats"]["mapping"] == 1 and r["stats"]["chunk"] == 4
        _same(ref, r, name)
        d.set_options(mapping=0)
        t = d.autotune()
        assert set(t["times_ms"]) == {f"warp,{k}" for k in (1, 2, 4, 8, 16)}
        d.close()
