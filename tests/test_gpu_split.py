"""The split of Alg. 5 (3D clipped diagrams) against the oracle.

With split = 1 the library first computes the restricted diagram on the
domain's boundary triangles; a site whose restricted cell there is empty and
that lies strictly inside a tetrahedron gets its whole Voronoi cell as one piece
(m, i), the others the per-tetrahedron pieces reached through negative flags.
The oracle knows nothing of the split: it clips every tetrahedron.  Per-site
measures, centroids and neighbours must match it as for split = 0; the pieces
of boundary sites must be the oracle's pieces, and a whole-cell piece must
carry exactly the bisector flags of the site's oracle pieces, none of which may
lie on the domain boundary."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_full, gpu_csr, gpu_run

pytestmark = pytest.mark.gpu

KEYS = ("measure", "centroid", "nbr_off", "nbr_idx")
SPLIT = dict(split=1, stats=1)


def _w(sites, verts, simp, name="case"):
    return dict(name=name, mode=4, sites=sites, verts=verts, simp=simp, f64=False)


def _check(w, options=SPLIT, meas_floor=0.0):
    d, r, p = gpu_run(w, options=options)
    assert r["status"] == 0 and r["stats"]["uncertain"] == 0
    op = O.Oracle(4, w["sites"], w["verts"], w["simp"]).enumerate()
    assert op.stats["uncertain"] == 0
    compare_full(w, r, p, op, meas_floor=meas_floor, split=True)
    # the pieces still partition the domain
    total = I.domain_measure(4, w["verts"], w["simp"])
    assert abs(float(p["measure"].double().sum()) - total) <= 1e-5 * total
    st = r["stats"]
    d.close()
    return st


def _two_cubes_on_an_edge():
    # two cubes of a 2x2x2 lattice that share one edge only: the boundary surface
    # has edges with four triangles (not a 2-manifold)
    return I.kuhn_lattice_tets(2, keep=lambda ix, iy, iz: (ix, iy, iz) in ((0, 0, 0), (1, 1, 0)))


@pytest.mark.parametrize("case,n,seed", [("cube6", 1, 61), ("cube6", 37, 62), ("lattice2", 3000, 63),
                                         ("shell8", 3000, 64), ("edge", 800, 65)])
def test_split_against_oracle(gpu, case, n, seed):
    if case == "cube6":
        v, s = I.cube_6tet()
        sites = I.uniform_sites(n, 3, I.SEED_BASE + seed)
    elif case == "lattice2":
        v, s = I.kuhn_lattice_tets(2)
        sites = I.uniform_sites(n, 3, I.SEED_BASE + seed)
    elif case == "shell8":
        v, s = I.small_shell(8)
        sites = I.shell_sites(n, seed=I.SEED_BASE + seed, ncomp=4)
    else:
        v, s = _two_cubes_on_an_edge()
        rng = np.random.default_rng(seed)
        sites = np.concatenate([rng.uniform(0.0, 0.5, (n // 2, 3)),
                                rng.uniform(0.0, 0.5, (n - n // 2, 3)) + [0.5, 0.5, 0.0]])
        sites = sites.astype(np.float32).astype(np.float64)
    st = _check(_w(sites, v, s))
    if n == 1:
        assert st["whole_cells"] == 0 and st["boundary_sites"] == 1  # the cell is the whole cube
    if n >= 800:
        assert st["whole_cells"] > 0 and st["boundary_sites"] > 0
        assert st["whole_cells"] + st["boundary_sites"] <= n


def test_split_sites_on_tetrahedron_faces(gpu):
    """Sites exactly on faces of the tetrahedra -- the cube faces x = 0.5 shared by
    two cells of the lattice, the diagonal faces x = y inside a cell, the domain
    boundary x = 0 -- and on the central mesh vertex: no tetrahedron holds them
    strictly, so they are computed per tetrahedron from every tetrahedron that
    may hold them.  Random coordinates in the face keep the configuration free of
    exact ties (symmetric sites would tie in Eq. 1 in any form)."""
    v, s = I.kuhn_lattice_tets(2)
    rng = np.random.default_rng(69)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    b, c = f32(rng.uniform(0.0, 1.0, (2, 80)))
    on_mid = np.stack([np.full(80, 0.5), b, c], 1)
    a, z = f32(rng.uniform(0.0, 0.5, (2, 80)))
    on_diag = np.stack([a, a, z], 1)
    b, c = f32(rng.uniform(0.0, 1.0, (2, 40)))
    on_bnd = np.stack([np.zeros(40), b, c], 1)
    sites = np.concatenate([on_mid, on_diag, on_bnd, [[0.5, 0.5, 0.5]], f32(rng.uniform(0.0, 1.0, (500, 3)))])
    sites = np.unique(sites, axis=0)
    st = _check(_w(sites, v, s))
    # at most the 500 random sites and none of those on a face can be whole cells
    assert 0 < st["whole_cells"] <= 500


def test_split_sites_outside_the_domain(gpu):
    """Sites over twice the cube's extent: cells reaching in from outside are
    boundary sites, cells missing the cube are empty with no pair at all."""
    v, s = I.cube_6tet()
    sites = I.uniform_sites(3000, 3, I.SEED_BASE + 66, lo=-0.5, hi=1.5)
    inside = np.all((sites >= 0.0) & (sites <= 1.0), axis=1).sum()
    st = _check(_w(sites, v, s), meas_floor=1.0 / max(1, int(inside)))
    assert st["whole_cells"] > 0


def test_split_matches_per_tet_and_learned_is_bitwise(gpu):
    """Shell, 30,000 clustered sites: neighbours of split = 0 and split = 1 are
    identical and measures agree within the tolerance; in split mode the learned
    form is bit-identical to the plain one."""
    v, s = I.small_shell(16)
    w = _w(I.shell_sites(30000, seed=I.SEED_BASE + 67, ncomp=8), v, s)
    d, per_tet, _ = gpu_run(w, options=dict(stats=1))
    d.set_options(**SPLIT)
    plain = d.compute()
    assert plain["status"] == 0 and plain["stats"]["whole_cells"] > 20000
    assert plain["stats"]["pairs"] < per_tet["stats"]["pairs"]
    assert torch.equal(plain["nbr_off"], per_tet["nbr_off"]) and torch.equal(plain["nbr_idx"], per_tet["nbr_idx"])
    rel = (plain["measure"].double() - per_tet["measure"].double()).abs() / per_tet["measure"].double()
    assert float(rel.max()) < 2e-5
    d.set_options(learned=1, topk=24, **SPLIT)
    lr = d.compute()
    for k in KEYS:
        assert torch.equal(plain[k], lr[k]), k
    d.close()


def test_split_lloyd_graph(gpu):
    v, s = I.small_shell(8)
    w = _w(I.shell_sites(5000, seed=I.SEED_BASE + 68, ncomp=4), v, s)
    from paper_2509_07175_b300 import binding as B
    a = B.diagram_from_workload(w, options=dict(split=1))
    b = B.diagram_from_workload(w, options=dict(split=1))
    a.lloyd(3, use_graph=True)
    b.lloyd(3, use_graph=False)
    assert torch.equal(a.sites(), b.sites())
    a.close()
    b.close()


