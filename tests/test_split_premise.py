"""The premise of the boundary / interior split (Alg. 5), checked with the oracle
alone (no GPU).

A site whose restricted cell on the domain's boundary triangles is empty (in
positive area) has its clipped cell equal to its whole Voronoi cell when the
site lies in the domain, and an empty clipped cell when it does not.  The
oracle computes all three independently: the clipped cells on the tetrahedra,
the restricted cells on the boundary triangles, and the whole cells clipped by
the mesh's bounding box (six tetrahedra).  On a domain with a hole and sites
inside, in the hole and outside it, every non-boundary site must satisfy the
premise, and the boundary sites must be exactly those whose clipped cell
differs from their whole cell."""
import numpy as np

import oracle as O
from paper_2509_07175_b300 import inputs as I


def _boundary_triangles(tets):
    faces = {}
    for a, t in enumerate(tets):
        for f in range(4):
            faces.setdefault(tuple(sorted(int(x) for k, x in enumerate(t) if k != f)), []).append(a)
    return np.array([k for k, v in faces.items() if len(v) == 1], dtype=np.int32)


def test_interior_cells_are_whole_cells():
    v, t = I.small_shell(8)
    rng = np.random.default_rng(5)
    inside = I.shell_sites(400, seed=I.SEED_BASE + 81, ncomp=3)
    around = rng.uniform(-1.2, 1.2, (120, 3))  # in the hole and outside the shell too
    sites = np.concatenate([inside, around]).astype(np.float32).astype(np.float64)
    n = len(sites)
    clipped = O.Oracle(4, sites, v, t).enumerate()
    cm, _, cnb = O.per_site(n, sites, clipped)
    surf = O.Oracle(3, sites, v, _boundary_triangles(t)).enumerate()
    sm, _, _ = O.per_site(n, sites, surf)
    lo, hi = v.min(0), v.max(0)
    bv, bt = I.kuhn_lattice_tets(1)
    bv = lo + bv * (hi - lo)
    whole = O.Oracle(4, sites, bv, bt).enumerate()
    wm, _, wnb = O.per_site(n, sites, whole)
    boundary = sm > 0
    assert 0 < boundary.sum() < n
    interior = ~boundary
    # interior sites: the clipped cell is the whole cell or nothing
    empty = cm[interior] == 0
    assert empty.any() and (~empty).any()
    full = np.flatnonzero(interior)[~empty]
    np.testing.assert_allclose(cm[full], wm[full], rtol=1e-10)
    assert all(cnb[i] == wnb[i] for i in full)
    # a site with an empty clipped cell and no boundary piece lies outside the shell
    r = np.linalg.norm(sites[np.flatnonzero(interior)[empty]], axis=1)
    assert ((r < 0.5) | (r > 0.99)).all()
    # boundary sites: their clipped cell is a proper part of the whole cell
    b = np.flatnonzero(boundary & (cm > 0))
    assert (cm[b] < wm[b] * (1 - 1e-9)).all()
