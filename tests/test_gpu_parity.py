"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: bit-exact neighbour sets and clip topology (the set of
non-empty (simplex, site) pieces and each piece's face flags); per-site
measures within 1e-5 relative; centroids within 1e-5 |c|.  Inputs are the
seeded generators of ``paper_2509_07175_b300.inputs``.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_full, compare_population, gpu_csr, gpu_run

pytestmark = pytest.mark.gpu


def _w(mode, sites, verts, simp, f64=False, name="case"):
    return dict(name=name, mode=mode, sites=sites, verts=verts, simp=simp, f64=f64)


def _full_check(w, brute=False, options=None, meas_floor=0.0):
    d, r, p = gpu_run(w, options=options)
    assert r["status"] == 0
    assert r["stats"]["uncertain"] == 0
    op = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"], brute=brute).enumerate()
    assert op.stats["uncertain"] == 0
    err = compare_full(w, r, p, op, meas_floor=meas_floor)
    # pieces partition each simplex
    per = np.zeros(len(w["simp"]))
    pm = p["measure"].double().cpu().numpy()
    np.add.at(per, p["simplex"].cpu().numpy(), pm)
    # FP32 pieces: error ~ u x (cell size) relative to each piece, so the check is
    # absolute, scaled by the mean cell measure |M| / n
    ref = I.simplex_measures(w["mode"], w["verts"], w["simp"])
    tol = 1e-5 * ref + 1e-5 * ref.sum() / len(w["sites"])
    assert (np.abs(per - ref) <= tol).all(), np.abs(per - ref).max()
    d.close()
    return err


def test_square_1000_fp64(gpu):
    """Config 1 at full size: unit square as 2 triangles, 1,000 uniform sites, FP64."""
    w = I.workload("square")
    err = _full_check(w)
    assert err["max_meas_rel"] < 1e-12


@pytest.mark.parametrize("n,seed", [(1, 5), (2, 6), (37, 7), (500, 8)])
def test_square_small_fp64(gpu, n, seed):
    v, s = I.square_grid_tris(3)
    w = _w(2, I.uniform_sites(n, 2, seed, f32=False), v, s, f64=True)
    _full_check(w)


def test_square_fp32(gpu):
    v, s = I.square_grid_tris(4)
    w = _w(2, I.uniform_sites(2000, 2, 9), v, s, f64=False)
    _full_check(w)


@pytest.mark.parametrize("dim,N", [(2, 8), (3, 4)])
def test_lattice_closed_form(gpu, dim, N):
    """Sites at box centres: cells are the boxes; exact ties resolve as inside."""
    sites = I.lattice_sites(N, dim)
    if dim == 2:
        v, s = I.square_2tri()
        w = _w(2, sites, v, s, f64=True)
    else:
        v, s = I.cube_6tet()
        w = _w(4, sites, v, s, f64=False)
    d, r, p = gpu_run(w)
    assert r["status"] == 0
    m = r["measure"].double().cpu().numpy()
    c = r["centroid"].double().cpu().numpy()
    assert np.abs(m - N ** -dim).max() <= 1e-6 * N ** -dim
    assert np.abs(c - sites).max() <= 1e-6
    nb = gpu_csr(r)
    idx = np.round(sites[:, :dim] * N - 0.5).astype(int)
    for i in range(len(sites)):
        exp = sorted(int(j) for j in np.nonzero(np.abs(idx - idx[i]).sum(axis=1) == 1)[0])
        assert nb[i] == exp


@pytest.mark.parametrize("n,seed,grid", [(1, 21, 1), (2, 22, 1), (300, 23, 1), (3000, 24, 2)])
def test_cube_small(gpu, n, seed, grid):
    v, s = I.kuhn_lattice_tets(grid)
    w = _w(4, I.uniform_sites(n, 3, seed), v, s)
    _full_check(w)


def test_shell_small_clustered(gpu):
    v, s = I.small_shell(8)
    w = _w(4, I.shell_sites(3000, seed=31, ncomp=4), v, s)
    _full_check(w)


def test_torus_small_surface(gpu):
    v, s = I.small_torus(60, 20)
    w = _w(3, I.surface_sites(1500, v, s, 41), v, s)
    _full_check(w)


def test_deterministic_bitwise(gpu):
    v, s = I.kuhn_lattice_tets(2)
    w = _w(4, I.uniform_sites(5000, 3, 51), v, s)
    d, r1, p1 = gpu_run(w)
    r2 = d.compute()
    for k in ("measure", "centroid", "nbr_off", "nbr_idx"):
        assert torch.equal(r1[k], r2[k]), k


KEYS = ("measure", "centroid", "nbr_off", "nbr_idx")
BENCH_FORM = dict(learned=1, topk=24, split=1, mapping=0)  # the form bench.py times (autotuned mapping)


def _population(name, forms):
    """Whole-population parity of a full-size workload: the oracle on every site,
    compared with each form's result; forms with the same split setting must
    also agree bit for bit (whole cells and per-tet pieces sum in different
    orders, so across that setting the oracle comparison is the bar)."""
    w = I.workload(name)
    op = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"]).all_sites()
    assert op.stats["uncertain"] == 0
    from paper_2509_07175_b300 import binding as B
    d = B.diagram_from_workload(w)
    errs, first = {}, {}
    for label, opts in forms:
        d.set_options(**opts)
        r = d.compute()
        assert r["status"] == 0
        sp = bool(opts.get("split"))
        if sp in first:  # bitwise against the first form of this split setting
            for k in KEYS:
                assert torch.equal(first[sp][k], r[k]), (label, k)
        else:
            first[sp] = r
            errs[label] = compare_population(w, r, d.pieces(), op, split=sp)
    d.close()
    print(name, errs)
    return errs


def test_cube_100k_full(gpu):
    """100,000 uniform sites in the 6-tet cube at full size, every site: the plain
    per-tetrahedron form and the learned + split form as timed against the
    oracle; the plain split form bit-identical to the timed one."""
    _population("cube", [("plain", dict()), ("bench", BENCH_FORM), ("plain_split", dict(split=1, mapping=1))])


def test_shell_1m_full(gpu):
    """1,000,000 clustered sites in the tetrahedralised shell (172,032 tets) at
    full size, every site: the plain per-tetrahedron form and the learned + split
    form as timed against the oracle; the plain split form bit-identical to the
    timed one."""
    _population("shell", [("plain", dict()), ("bench", BENCH_FORM), ("plain_split", dict(split=1, mapping=1))])


@pytest.mark.parametrize("name,n", [("cube", 20000), ("shell", 30000), ("square", 1000), ("torus", 20000)])
def test_learned_form_equals_plain_bitwise(gpu, name, n):
    """The learned proposal only orders and shortcuts the search; every clip is
    still decided by the exact test and integration is canonical, so the output
    equals the plain search's bit for bit (per-site measure, centroid, CSR)."""
    w = I.workload(name, n=n)
    d = None
    from paper_2509_07175_b300 import binding as B
    d = B.diagram_from_workload(w)
    plain = d.compute()
    for k in (8, 16, 32):
        for nearest in (32, 64):  # lists of the 32 nearest, or extended to the 64 nearest
            d.set_options(learned=1, topk=k, stats=1, mapping=1, nearest=nearest)
            lr = d.compute()
            assert lr["stats"]["learned_hits"] > 0 and lr["stats"]["nearest"] == nearest
            for key in ("measure", "centroid", "nbr_off", "nbr_idx"):
                assert torch.equal(plain[key], lr[key]), (k, nearest, key)
    d.close()


@pytest.mark.parametrize("mode", [2, 4])
def test_coincident_sites_are_reported(gpu, mode):
    """Two equal sites have no bisector and Eq. 1 would give both the same cell:
    the compute reports VD_ERR_DUPLICATE instead of a double cover."""
    from paper_2509_07175_b300 import binding as B
    if mode == 2:
        v, s = I.square_grid_tris(2)
        sites = I.uniform_sites(200, 2, I.SEED_BASE + 0x170, f32=False)
        f64 = True
    else:
        v, s = I.cube_6tet()
        sites = I.uniform_sites(500, 3, I.SEED_BASE + 0x171)
        f64 = False
    sites[7] = sites[123]
    w = _w(mode, sites, v, s, f64=f64)
    d = B.diagram_from_workload(w)
    with pytest.raises(B.VDError) as e:
        d.compute()
    assert e.value.code == -9
    sites[7, 0] = np.nextafter(np.float32(sites[7, 0]), np.float32(2)) if not f64 else np.nextafter(sites[7, 0], 2)
    d.update_sites(torch.tensor(sites[:, :2 if mode == 2 else 3], dtype=torch.float64 if f64 else torch.float32,
                                device="cuda"))
    r = d.compute()   # one ulp apart: a valid, if thin, pair of cells
    assert r["status"] == 0
    d.close()


def test_cube2m_full(gpu):
    """Config 5 at full size, every site: 2,000,000 uniform sites in the 6-tet cube
    (learned + split as timed), and the learned form with a network ranking
    (untrained) bit-identical to it."""
    from paper_2509_07175_b300 import binding as B
    _population("cube2m", [("bench", BENCH_FORM)])
    w = I.workload("cube2m")
    d = B.diagram_from_workload(w, options=BENCH_FORM)
    r = d.compute()
    d.mlp_init(9)
    d.set_options(proposal=B.PROPOSAL_MLP, **BENCH_FORM)
    lr = d.compute()
    for key in KEYS:
        assert torch.equal(r[key], lr[key]), key
    d.close()


@pytest.mark.parametrize("mode,n,seed", [(4, 3000, 51), (2, 1500, 52), (3, 1200, 53)])
def test_sites_outside_the_domain(gpu, mode, n, seed):
    """Sites spread over twice the domain's extent: many have no simplex of their
    own (no site seed), some cells are empty, others reach into the domain from
    outside; the pieces must still match the oracle."""
    if mode == 4:
        v, s = I.cube_6tet()
        sites = I.uniform_sites(n, 3, I.SEED_BASE + seed, lo=-0.5, hi=1.5)
    elif mode == 2:
        v, s = I.square_grid_tris(4)
        sites = I.uniform_sites(n, 2, I.SEED_BASE + seed, lo=-0.5, hi=1.5)
    else:
        v, s = I.small_torus()
        sites = I.uniform_sites(n, 3, I.SEED_BASE + seed, lo=-1.6, hi=1.6)
    w = _w(mode, sites, v, s)
    # cells reaching in from outside can be slivers far from their site: measures
    # are checked relative to max(m, mean cell measure), the mean taken over the
    # sites inside the domain's bounding box
    lo, hi = v.min(axis=0), v.max(axis=0)
    dim = 2 if mode == 2 else 3
    inside = np.all((sites[:, :dim] >= lo[:dim]) & (sites[:, :dim] <= hi[:dim]), axis=1).sum()
    _full_check(w, meas_floor=I.domain_measure(mode, v, s) / max(1, int(inside)))
    d, r, _ = gpu_run(w)
    assert (r["measure"] == 0).any()   # some cells miss the domain entirely
    d.close()
