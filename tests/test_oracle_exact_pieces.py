"""The oracle's pieces against exact rational arithmetic (brute force over all
triples of planes, tests/exact_pieces.py): which pieces have positive volume and
which of their faces have positive area (Sec. 2.2), on tiny inputs where every
site's bisector is used, and on the slivers of the 1M-site shell workload that
float64 integration cannot resolve."""
import numpy as np
import pytest

import oracle as O
from paper_2509_07175_b300 import inputs as I
from exact_pieces import candidates, piece


def _oracle_pieces(op):
    out = {}
    for k in range(len(op.a)):
        if op.meas[k] > 0:
            fl = op.flags[op.foff[k]:op.foff[k + 1]]
            out[(int(op.a[k]), int(op.i[k]))] = (set(int(x) for x in fl if x >= 0), int((fl < 0).sum()))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_cube_every_piece(seed):
    """10 uniform sites in the 6-tetrahedra cube: every (tet, site) pair computed
    exactly from all 9 bisectors and the 4 tet faces."""
    v, s = I.cube_6tet()
    sites = I.uniform_sites(10, 3, I.SEED_BASE + 0x7E0 + seed).astype(np.float64)
    got = _oracle_pieces(O.Oracle(4, sites, v, s).enumerate())
    want = {}
    for a in range(len(s)):
        for i in range(len(sites)):
            pos, faces, ntet, _ = piece(v[s[a]], sites[i], [(j, sites[j]) for j in range(len(sites)) if j != i])
            if pos:
                want[(a, i)] = (faces, ntet)
    assert set(got) == set(want)
    for k in want:
        assert got[k] == want[k], (k, got[k], want[k])


def test_kuhn_lattice_pieces():
    """A 2x2x2 Kuhn lattice (48 tets) with 12 sites: every pair, exactly."""
    v, s = I.kuhn_lattice_tets(2)
    sites = I.uniform_sites(12, 3, I.SEED_BASE + 0x7E9).astype(np.float64)
    got = _oracle_pieces(O.Oracle(4, sites, v, s).enumerate())
    want = {}
    for a in range(len(s)):
        for i in range(len(sites)):
            pos, faces, ntet, _ = piece(v[s[a]], sites[i], [(j, sites[j]) for j in range(len(sites)) if j != i])
            if pos:
                want[(a, i)] = (faces, ntet)
    assert set(got) == set(want)
    for k in want:
        assert got[k] == want[k], (k, got[k], want[k])


@pytest.fixture(scope="module")
def shell():
    return I.workload("shell")


# pieces of site 913097 of the 1M-site shell workload: (15714) a sliver whose
# corners differ by ~3e-8 (volume ~1e-23, below float64's resolution of its
# integration), (15716) one of volume ~1e-23 that float64 happens to resolve
@pytest.mark.parametrize("a", [15714, 15716])
def test_shell_slivers(shell, a):
    w = shell
    sites = np.asarray(w["sites"], np.float64)
    i = 913097
    others, excluded = candidates(sites, i, 30)
    pos, faces, ntet, reach = piece(np.asarray(w["verts"], np.float64)[w["simp"][a]], sites[i], others)
    assert 2 * reach * (1 + 1e-9) < excluded  # no site beyond the 30 nearest can cut it
    assert pos
    got = _oracle_pieces(O.Oracle(4, w["sites"], w["verts"], w["simp"]).site_pieces(np.array([i])))
    assert got[(a, i)] == (faces, ntet)


@pytest.mark.parametrize("seed", [1, 2])
def test_tiny_square_every_piece(seed):
    """2D: 12 uniform FP64 sites in the unit square as 2 triangles, every
    (triangle, site) pair computed exactly from all 11 bisectors and the 3 edges."""
    from exact_pieces import polygon_piece
    v, s = I.square_grid_tris(1)
    sites = I.uniform_sites(12, 2, I.SEED_BASE + 0x7F0 + seed, f32=False)
    got = _oracle_pieces(O.Oracle(2, sites, v, s).enumerate())
    want = {}
    for a in range(len(s)):
        for i in range(len(sites)):
            pos, edges, ntri = polygon_piece(v[s[a]], sites[i], [(j, sites[j]) for j in range(len(sites)) if j != i])
            if pos:
                want[(a, i)] = (edges, ntri)
    assert set(got) == set(want)
    for k in want:
        assert got[k] == want[k], (k, got[k], want[k])


def test_tiny_surface_every_piece():
    """Surface: 10 sites jittered off a small torus mesh (240 triangles), every
    (triangle, site) pair computed exactly in the triangle's plane."""
    from exact_pieces import surface_piece
    v, s = I.torus_domain(nu=12, nv=10)
    sites = I.surface_sites(10, v, s, I.SEED_BASE + 0x7F8)
    got = _oracle_pieces(O.Oracle(3, sites, v, s).enumerate())
    want = {}
    for a in range(len(s)):
        for i in range(len(sites)):
            pos, edges, ntri = surface_piece(v[s[a]], sites[i], [(j, sites[j]) for j in range(len(sites)) if j != i])
            if pos:
                want[(a, i)] = (edges, ntri)
    assert set(got) == set(want)
    for k in want:
        assert got[k] == want[k], (k, got[k], want[k])
