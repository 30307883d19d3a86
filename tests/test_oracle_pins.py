"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

The oracle (``oracle/``) computes every piece P_{a,i} = T_a cap Omega_i from
Eq. 1 (Sec. 2.1) with the face flags of Sec. 2.2.  These tests tie it to
things other than itself:

* brute force: clipping by all n-1 bisectors (no pruning, no kd-tree) must give
  the same pieces as the security-radius form;
* closed forms: lattice sites give lattice boxes, one site gives the domain,
  two sites give a half-space cut (tests/golden/closed_forms.json);
* invariants: the pieces partition every simplex (Sec. 2.1: the cells
  partition the domain), neighbour relations are symmetric and the shared face
  has the same measure seen from both sides;
* statistics: mean degree of interior cells of uniform sites (6 in 2D,
  2 + 48 pi^2 / 35 ~ 15.54 in 3D, Poisson-Voronoi).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2509_07175_b300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _domain(mode, name="unit"):
    if mode == 2:
        return I.square_2tri()
    if mode == 4:
        return I.cube_6tet()
    raise ValueError(mode)


def _compare(pa, pb, tol=1e-12):
    ta, tb = pa.topology(), pb.topology()
    assert ta == tb
    ma = {(int(a), int(i)): (m, m1) for a, i, m, m1 in zip(pa.a, pa.i, pa.meas, pa.m1) if m > 0}
    mb = {(int(a), int(i)): (m, m1) for a, i, m, m1 in zip(pb.a, pb.i, pb.meas, pb.m1) if m > 0}
    for k in ma:
        assert abs(ma[k][0] - mb[k][0]) <= tol * max(1.0, abs(ma[k][0]))
        assert np.abs(ma[k][1] - mb[k][1]).max() <= tol


@pytest.mark.parametrize("mode,n,seed", [(2, 150, 11), (4, 120, 12), (3, 80, 13), (2, 40, 14), (4, 60, 15)])
def test_brute_force_equals_security_radius(mode, n, seed):
    if mode == 3:
        v, s = I.small_torus(24, 8)
        sites = I.surface_sites(n, v, s, seed)
    elif mode == 2:
        v, s = I.square_grid_tris(3)
        sites = I.uniform_sites(n, 2, seed, f32=False)
    else:
        v, s = I.kuhn_lattice_tets(2)
        sites = I.uniform_sites(n, 3, seed)
    pb = O.Oracle(mode, sites, v, s, brute=True).enumerate()
    ps = O.Oracle(mode, sites, v, s, brute=False).enumerate()
    assert pb.stats["uncertain"] == 0 and ps.stats["uncertain"] == 0
    assert pb.stats["error"] == 0 and ps.stats["error"] == 0
    _compare(pb, ps)


def test_brute_force_small_shell():
    v, s = I.small_shell(6)
    sites = I.shell_sites(60, seed=77, ncomp=3)
    pb = O.Oracle(4, sites, v, s, brute=True).enumerate()
    ps = O.Oracle(4, sites, v, s, brute=False).enumerate()
    _compare(pb, ps)
    assert abs(ps.meas.sum() - I.domain_measure(4, v, s)) < 1e-12


@pytest.mark.parametrize("dim,N,grid", [(2, 4, 1), (2, 8, 1), (2, 4, 3), (3, 4, 1), (3, 2, 3), (3, 4, 3)])
def test_lattice_closed_form(dim, N, grid):
    """Sites at box centres (k+1/2)/N: each cell is its box, of measure N^-d, with
    centroid at the site; neighbours are the 2d axis-adjacent sites.  Corner- and
    edge-adjacent sites touch with zero measure and are not neighbours.  The mesh
    is chosen so that no Voronoi face lies inside a mesh face (there the tie rule
    keeps the mesh face and its simplex flag, and no bisector clip happens).
    Mesh coordinates are dyadic so that every tie is exactly representable."""
    sites = I.lattice_sites(N, dim)
    ticks = None if grid == 1 else [0.0, 0.375, 0.625, 1.0]
    if dim == 2:
        v, s = I.square_grid_tris(grid, ticks=ticks)
        mode = 2
    else:
        v, s = I.kuhn_lattice_tets(grid, ticks=ticks)
        mode = 4
    for brute in (True, False):
        p = O.Oracle(mode, sites, v, s, brute=brute).enumerate()
        assert p.stats["uncertain"] == 0 and p.stats["error"] == 0
        meas, cen, nb = O.per_site(len(sites), sites, p)
        assert np.abs(meas - N ** -dim).max() < 1e-15
        assert np.abs(cen - sites).max() < 1e-15
        idx = np.round(sites[:, :dim] * N - 0.5).astype(int)
        for i in range(len(sites)):
            exp = sorted(int(j) for j in np.nonzero(np.abs(idx - idx[i]).sum(axis=1) == 1)[0])
            assert nb[i] == exp


@pytest.mark.parametrize("case", ["two_sites_square_axis", "two_sites_square_diag", "two_sites_cube_diag",
                                  "two_sites_cube_axis", "one_site_square", "one_site_cube"])
def test_golden_closed_forms(case):
    g = json.load(open(GOLD))[case]
    v, s = _domain(g["mode"])
    sites = np.array(g["sites"], dtype=np.float64)
    for brute in (True, False):
        p = O.Oracle(g["mode"], sites, v, s, brute=brute).enumerate()
        meas, cen, _ = O.per_site(len(sites), sites, p)
        np.testing.assert_allclose(meas, g["measure"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(cen, g["centroid"], rtol=0, atol=1e-14)


def test_one_site_surface_is_whole_mesh():
    v, s = I.small_torus(16, 6)
    sites = np.array([[1.3, 0.0, 0.0]])
    p = O.Oracle(3, sites, v, s).enumerate()
    a, b, c = v[s[:, 0]], v[s[:, 1]], v[s[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    cen = (area[:, None] * (a + b + c) / 3).sum(0) / area.sum()
    meas, c2, _ = O.per_site(1, sites, p)
    assert abs(meas[0] - area.sum()) < 1e-12
    assert np.abs(c2[0] - cen).max() < 1e-12
    assert len(p) == len(s) and (p.meas > 0).all()


@pytest.mark.parametrize("mode,n,seed", [(2, 400, 21), (4, 300, 22), (3, 300, 23)])
def test_partition_and_symmetry(mode, n, seed):
    if mode == 3:
        v, s = I.small_torus(40, 12)
        sites = I.surface_sites(n, v, s, seed)
    elif mode == 2:
        v, s = I.square_2tri()
        sites = I.uniform_sites(n, 2, seed, f32=False)
    else:
        v, s = I.cube_6tet()
        sites = I.uniform_sites(n, 3, seed)
    p = O.Oracle(mode, sites, v, s).enumerate()
    assert p.stats["uncertain"] == 0 and p.stats["error"] == 0
    # pieces partition each simplex
    per_simplex = np.zeros(len(s))
    np.add.at(per_simplex, p.a, p.meas)
    np.testing.assert_allclose(per_simplex, I.simplex_measures(mode, v, s), rtol=1e-12)
    # every site with a non-empty cell appears; the neighbour relation is symmetric
    meas, cen, nb = O.per_site(len(sites), sites, p)
    for i in range(len(sites)):
        for j in nb[i]:
            assert i in nb[j]
    # a bisector face has the same measure seen from both of its cells
    face = {}
    for q in range(len(p)):
        if p.meas[q] <= 0:
            continue
        for f, fm in zip(p.face_flags(q), p.face_measures(q)):
            if f >= 0:
                face[(int(p.a[q]), int(p.i[q]), int(f))] = fm
    for (a, i, j), fm in face.items():
        assert abs(face[(a, j, i)] - fm) <= 1e-9 * max(fm, 1e-300) + 1e-15
    # simplex faces: the piece of site i on the face shared by T_a and T_b is mirrored
    for q in range(len(p)):
        if p.meas[q] <= 0:
            continue
        for f in p.face_flags(q):
            if f < 0 and f != O.FLAG_BOUNDARY:
                b = -int(f) - 1
                assert (b, int(p.i[q])) in p.topology()


def test_site_flood_matches_enumeration():
    v, s = I.small_shell(6)
    sites = I.shell_sites(300, seed=91, ncomp=4)
    o = O.Oracle(4, sites, v, s)
    full = o.enumerate()
    pick = np.arange(0, 300, 7)
    sub = o.site_pieces(pick)
    tf = {k: t for k, t in full.topology().items() if k[1] in set(pick.tolist())}
    assert sub.topology() == tf


def test_mean_degree_statistics():
    """Interior cells of uniform (Poisson) sites: mean degree 6 in 2D and
    2 + 48 pi^2/35 = 15.535... in 3D.  Loose statistical check."""
    sites = I.uniform_sites(3000, 2, 31, f32=False)
    v, s = I.square_2tri()
    p = O.Oracle(2, sites, v, s).enumerate()
    _, _, nb = O.per_site(len(sites), sites, p)
    inner = np.all((sites[:, :2] > 0.15) & (sites[:, :2] < 0.85), axis=1)
    deg2 = np.mean([len(nb[i]) for i in np.nonzero(inner)[0]])
    assert abs(deg2 - 6.0) < 0.1
    sites = I.uniform_sites(3000, 3, 32)
    v, s = I.cube_6tet()
    p = O.Oracle(4, sites, v, s).enumerate()
    _, _, nb = O.per_site(len(sites), sites, p)
    inner = np.all((sites > 0.25) & (sites < 0.75), axis=1)
    deg3 = np.mean([len(nb[i]) for i in np.nonzero(inner)[0]])
    assert abs(deg3 - (2 + 48 * np.pi ** 2 / 35)) < 0.6


def test_planted_mistake_is_caught():
    """A plausible slip in the oracle -- the bisector offset |w|^2/2 replaced by
    |w|^2 -- must break the two-site closed form.  The slip is planted in a copy
    of the oracle source compiled on the CPU."""
    import subprocess
    import tempfile
    import ctypes
    src = open(os.path.join(os.path.dirname(O.__file__), "vd_oracle.c")).read()
    bad = src.replace("*c = S##_scale(S##_dot3(n, n), 0.5);", "*c = S##_scale(S##_dot3(n, n), 1.0);")
    assert bad != src
    with tempfile.TemporaryDirectory() as d:
        cpath, lpath = os.path.join(d, "bad.c"), os.path.join(d, "libbad.so")
        open(cpath, "w").write(bad)
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", lpath, cpath, "-lpthread", "-lm"])
        saved = O._lib
        try:
            O._lib = None
            lib = ctypes.CDLL(lpath)
            P = ctypes.c_void_p
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, P,
                                       ctypes.c_int, ctypes.c_int]
            lib.orc_enumerate.restype = ctypes.POINTER(O._Result)
            lib.orc_enumerate.argtypes = [P]
            lib.orc_free_result.argtypes = [ctypes.POINTER(O._Result)]
            lib.orc_destroy.argtypes = [P]
            lib.orc_adjacency.argtypes = [P, P]
            lib.orc_pieces.restype = ctypes.POINTER(O._Result)
            lib.orc_site_pieces.restype = ctypes.POINTER(O._Result)
            O._lib = lib
            g = json.load(open(GOLD))["two_sites_cube_axis"]
            v, s = _domain(4)
            sites = np.array(g["sites"])
            p = O.Oracle(4, sites, v, s, brute=True).enumerate()
            meas, _, _ = O.per_site(2, sites, p)
            assert np.abs(meas - np.array(g["measure"])).max() > 1e-3
        finally:
            O._lib = saved


# ----- power diagrams (power distance |x - v_i|^2 - w_i) ---------------------------

def _power_case(mode, n, seed):
    v, s = _domain(mode)
    dim = 2 if mode == 2 else 3
    sites = I.uniform_sites(n, dim, seed, f32=False)
    measure = I.domain_measure(mode, v, s)
    rng = np.random.default_rng(seed)
    w = rng.uniform(-measure / n, measure / n, n)  # the paper's weight range
    return v, s, sites, w


@pytest.mark.parametrize("mode,n", [(2, 120), (4, 60)])
def test_power_equal_weights_is_voronoi(mode, n):
    # equal weights cancel in every power bisector: the power diagram is the Voronoi diagram
    v, s, sites, _ = _power_case(mode, n, 21)
    pv = O.Oracle(mode, sites, v, s).enumerate()
    pw = O.Oracle(mode, sites, v, s, weights=np.full(n, 0.37)).enumerate()
    _compare(pv, pw, tol=1e-12)


def _two_site_power(mode, dw, oracle_mod=O):
    # two sites on a line parallel to an axis, 0.5 apart, weights 0 and dw: the power
    # bisector is the plane x* = (x2^2 - x1^2 - dw) / (2 (x2 - x1)) = 0.5 - dw
    v, s = _domain(mode)
    sites = np.array([[0.25, 0.5, 0.0], [0.75, 0.5, 0.0]]) if mode == 2 else \
        np.array([[0.5, 0.5, 0.25], [0.5, 0.5, 0.75]])
    p = oracle_mod.Oracle(mode, sites, v, s, brute=True, weights=np.array([0.0, dw])).enumerate()
    meas, cen, nb = oracle_mod.per_site(2, sites, p)
    return meas, cen, nb


@pytest.mark.parametrize("mode", [2, 4])
@pytest.mark.parametrize("dw", [0.0, 0.1, -0.2, 0.3, 0.8])
def test_power_two_sites_closed_form(mode, dw):
    meas, cen, nb = _two_site_power(mode, dw)
    xs = 0.5 - dw
    if xs <= 0:  # site 0 is dominated everywhere: empty cell
        assert meas[0] == 0 and nb[0] == [] and abs(meas[1] - 1.0) < 1e-12
        return
    assert abs(meas[0] - xs) < 1e-12 and abs(meas[1] - (1 - xs)) < 1e-12
    ax = 0 if mode == 2 else 2
    assert abs(cen[0][ax] - xs / 2) < 1e-12 and abs(cen[1][ax] - (1 + xs) / 2) < 1e-12
    assert nb[0] == [1] and nb[1] == [0]


@pytest.mark.parametrize("mode,n,seed", [(2, 150, 31), (4, 80, 32), (2, 60, 33)])
def test_power_brute_equals_security_radius(mode, n, seed):
    v, s, sites, w = _power_case(mode, n, seed)
    pb = O.Oracle(mode, sites, v, s, brute=True, weights=w).enumerate()
    ps = O.Oracle(mode, sites, v, s, brute=False, weights=w).enumerate()
    _compare(pb, ps)
    # the cells still partition the domain
    total = I.domain_measure(mode, v, s)
    assert abs(pb.meas.sum() - total) < 1e-12 * max(1.0, total) * 10


def test_power_planted_sign_flip_is_caught():
    """The weight difference with the wrong sign in the power bisector must break the
    two-site closed form (planted in a copy of the oracle source, compiled on the CPU)."""
    import ctypes
    import subprocess
    import tempfile
    src = open(os.path.join(os.path.dirname(O.__file__), "vd_oracle.c")).read()
    bad = src.replace("S##_sub(S##_c(C->w[p->a]), S##_c(C->w[site]))", "S##_sub(S##_c(C->w[site]), S##_c(C->w[p->a]))")
    assert bad != src
    with tempfile.TemporaryDirectory() as d:
        cpath, lpath = os.path.join(d, "bad.c"), os.path.join(d, "libbad.so")
        open(cpath, "w").write(bad)
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", lpath, cpath, "-lpthread", "-lm"])
        saved = O._lib
        try:
            O._lib = None
            lib = ctypes.CDLL(lpath)
            P = ctypes.c_void_p
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, P,
                                       ctypes.c_int, ctypes.c_int]
            lib.orc_set_weights.argtypes = [P, P]
            lib.orc_set_weights.restype = None
            lib.orc_enumerate.restype = ctypes.POINTER(O._Result)
            lib.orc_enumerate.argtypes = [P]
            lib.orc_free_result.argtypes = [ctypes.POINTER(O._Result)]
            lib.orc_destroy.argtypes = [P]
            O._lib = lib
            meas, _, _ = _two_site_power(2, 0.1)
            assert abs(meas[0] - 0.4) > 1e-3
        finally:
            O._lib = saved


# ----- power diagrams restricted to a surface (mode 3) -----------------------------

def _surface_power_case(n, seed):
    v, s = I.torus_domain(nu=36, nv=12)
    sites = I.surface_sites(n, v, s, seed)
    measure = I.domain_measure(3, v, s)
    rng = np.random.default_rng(seed)
    return v, s, sites, rng.uniform(-measure / n, measure / n, n)


def test_power_surface_equal_weights_is_voronoi():
    """Equal weights cancel in every power bisector, on a surface too."""
    v, s, sites, _ = _surface_power_case(90, 41)
    pv = O.Oracle(3, sites, v, s).enumerate()
    pw = O.Oracle(3, sites, v, s, weights=np.full(len(sites), -0.21)).enumerate()
    _compare(pv, pw, tol=1e-12)


@pytest.mark.parametrize("n,seed", [(70, 42), (40, 43)])
def test_power_surface_brute_equals_security_radius(n, seed):
    """Restricted power diagram on a torus: all n-1 power bisectors against the
    generalised security radius, and the cells partition the surface."""
    v, s, sites, w = _surface_power_case(n, seed)
    pb = O.Oracle(3, sites, v, s, brute=True, weights=w).enumerate()
    ps = O.Oracle(3, sites, v, s, brute=False, weights=w).enumerate()
    _compare(pb, ps)
    total = I.domain_measure(3, v, s)
    assert abs(pb.meas.sum() - total) < 1e-10 * total


@pytest.mark.parametrize("e1,e2,dw", [(0.0, 0.0, 0.1), (0.1, 0.0, 0.0), (0.05, 0.2, -0.1), (0.3, 0.1, 0.2)])
def test_power_surface_two_sites_off_the_plane(e1, e2, dw):
    """A planar square mesh (z = 0) in surface mode, two sites at heights e1, e2
    above it with weights 0 and dw: on the plane the power distance of site i is
    (x - x_i)^2 + (y - 1/2)^2 + e_i^2 - w_i, so the cells meet on the line
    x* = 1/2 - dw + e2^2 - e1^2 (sites at x = 1/4 and 3/4)."""
    v, s = I.square_2tri()
    sites = np.array([[0.25, 0.5, e1], [0.75, 0.5, e2]])
    p = O.Oracle(3, sites, v, s, brute=True, weights=np.array([0.0, dw])).enumerate()
    meas, cen, nb = O.per_site(2, sites, p)
    xs = 0.5 - dw + e2 ** 2 - e1 ** 2
    assert 0 < xs < 1
    assert abs(meas[0] - xs) < 1e-12 and abs(meas[1] - (1 - xs)) < 1e-12
    assert abs(cen[0][0] - xs / 2) < 1e-12 and abs(cen[1][0] - (1 + xs) / 2) < 1e-12
    assert abs(cen[0][2]) < 1e-12 and abs(cen[1][2]) < 1e-12   # centroids lie on the surface
    assert nb[0] == [1] and nb[1] == [0]


@pytest.mark.parametrize("mode", [2, 3, 4])
def test_all_sites_equals_enumeration(mode):
    """The per-site form over every site (used for whole-population checks at full
    size, parallel over sites) gives exactly the pieces of the per-simplex form."""
    if mode == 2:
        v, s = I.square_grid_tris(3)
        sites = I.uniform_sites(400, 2, 95, f32=False)
    elif mode == 3:
        v, s = I.torus_domain(nu=30, nv=10)
        sites = I.surface_sites(300, v, s, 96)
    else:
        v, s = I.kuhn_lattice_tets(2)
        sites = I.uniform_sites(500, 3, 97)
    o = O.Oracle(mode, sites, v, s)
    a, b = o.enumerate(), o.all_sites()
    _compare(a, b, tol=0.0)
