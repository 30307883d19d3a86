"""The paper's serial method (Alg. 1 + Alg. 2, real edges, the queue over
positive flags and the intermediate polytope G_{a,j}) against the FP64 oracle.

Bar: the same non-empty pieces with the same face flags (bit-exact topology),
per-site measures and centroids within 1e-12 relative (both sides are FP64, by
different algorithms), per-piece measures within 1e-12 of the mean cell
measure, and every clip of Alg. 1 leaving a face on the final piece
(Sec. 3.3: "all the clippings are contributed to the final result")."""
import numpy as np
import pytest

import oracle as O
from paper_2509_07175_b300 import inputs as I
from paper_2509_07175_b300 import serial as S


def _check(mode, sites, verts, simp):
    r = S.Serial(mode, sites, verts, simp).run()
    assert r.status == 0 and r.stats["errors"] == 0
    assert r.stats["uncertain"] == 0
    op = O.Oracle(mode, sites, verts, simp).enumerate()
    gt, ot = r.topology(), op.topology()
    assert set(gt) == set(ot), (sorted(set(ot) - set(gt))[:5], sorted(set(gt) - set(ot))[:5])
    bad = [k for k in ot if ot[k] != gt[k]]
    assert not bad, (bad[0], ot[bad[0]], gt[bad[0]])
    n = len(sites)
    om, oc, onb = O.per_site(n, sites, op)
    sm = np.zeros(n)
    sc = np.zeros((n, 3))
    np.add.at(sm, r.i, r.meas)
    np.add.at(sc, r.i, r.m1)
    ok = om > 0
    assert ((sm > 0) == ok).all()
    assert (np.abs(sm[ok] - om[ok]) <= 1e-12 * om[ok]).all(), (np.abs(sm[ok] - om[ok]) / om[ok]).max()
    cen = sites.copy()
    cen[ok] += sc[ok] / sm[ok, None]
    assert (np.linalg.norm(cen - oc, axis=1) <= 1e-12 * np.linalg.norm(oc, axis=1)).all()
    # pieces: the same measures, up to 1e-12 of the mean cell
    omap = {(int(a), int(i)): m for a, i, m in zip(op.a, op.i, op.meas) if m > 0}
    smap = {(int(a), int(i)): m for a, i, m in zip(r.a, r.i, r.meas) if m > 0}
    scale = om.sum() / n
    assert max(abs(smap[k] - omap[k]) for k in omap) <= 1e-12 * scale
    # Sec. 3.3: every clip of Alg. 1 contributes a face
    assert r.stats["excess_clips"] == 0 and r.stats["fallback"] == 0
    assert r.stats["bisector_faces"] >= r.stats["clips"]
    return r


def test_square_config1():
    """2D: unit square as 2 triangles, 1,000 uniform FP64 sites."""
    w = I.workload("square")
    _check(w["mode"], w["sites"], w["verts"], w["simp"])


@pytest.mark.parametrize("n,seed", [(1, 11), (2, 12), (40, 13)])
def test_square_small(n, seed):
    v, s = I.square_grid_tris(3)
    _check(2, I.uniform_sites(n, 2, seed, f32=False), v, s)


def test_cube():
    """3D: the unit cube as 6 tetrahedra, 5,000 uniform sites."""
    w = I.workload("cube", n=5000)
    _check(w["mode"], w["sites"], w["verts"], w["simp"])


def test_cube_lattice_mesh():
    """3D: a 3x3x3 Kuhn lattice of tetrahedra (162), 2,000 sites."""
    v, s = I.kuhn_lattice_tets(3)
    _check(4, I.uniform_sites(2000, 3, I.SEED_BASE + 0x401), v, s)


def test_shell():
    """3D: a smaller tetrahedralised spherical shell with clustered sites."""
    v, s = I.shell_domain(ncube=8)
    _check(4, I.shell_sites(4000, I.SEED_BASE + 0x402), v, s)


def test_torus():
    """Surface: a torus triangle mesh, sites on it jittered off the surface."""
    v, s = I.torus_domain(nu=80, nv=20)
    _check(3, I.surface_sites(3000, v, s, I.SEED_BASE + 0x403), v, s)


def test_rejects_bad_mesh():
    v, s = I.kuhn_lattice_tets(2)
    bad = s.copy()
    bad[0, 0] = len(v)
    with pytest.raises(ValueError):
        S.Serial(4, I.uniform_sites(10, 3, 1), v, bad)
    with pytest.raises(ValueError):
        S.Serial(4, I.uniform_sites(10, 3, 1), v, np.concatenate([s, s[:1]]))
