"""Power diagrams in 3D (tetrahedral meshes, the box form) and restricted to a
surface (the torus), against the weighted oracle (Sec. 6.3: the sites lifted one
dimension up, the clipped / restricted diagram of the lifted sites).

The library lifts site i to (v_i, h_i), h_i = sqrt(eta - w_i) in float32 with
eta = max w; the weights it realises are eta - h_i^2 exactly, and a constant
shift of all weights changes nothing, so the oracle is given -h_i^2 computed
here from the same float32 arithmetic (IEEE subtraction and square root).
Topology and neighbours are compared exactly, measures within 1e-5 of
max(m, |M| / n): a power cell far smaller than the lift height carries an FP32
error scaled by the typical cell."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_population

pytestmark = pytest.mark.gpu

KEYS = ("measure", "centroid", "nbr_off", "nbr_idx")


def _weights(n, measure, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, n) * spread * measure / n).astype(np.float32)


def _realised(w):
    wf = w.astype(np.float32)
    h = np.sqrt(np.float32(wf.max()) - wf)          # float32, as on the device
    return -(h.astype(np.float64) ** 2)


def _check(w, weights, options=None, brute=False, box=False):
    d = B.diagram_from_workload(w, options=options)
    d.set_weights(torch.tensor(weights, device="cuda"))
    r = d.compute()
    assert r["status"] == 0 and r["stats"]["uncertain"] == 0
    op = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"], brute=brute, weights=_realised(weights)).enumerate()
    assert op.stats["uncertain"] == 0
    measure = I.domain_measure(w["mode"], w["verts"], w["simp"])
    err = compare_population(w, r, d.pieces(), op, box=box, meas_floor=measure / len(w["sites"]))
    assert abs(float(r["measure"].double().sum()) - measure) < 1e-5 * measure
    return d, r, err


@pytest.mark.parametrize("n,seed,spread,brute", [(200, 61, 1.0, True), (3000, 62, 1.0, False),
                                                 (3000, 63, 6.0, False)])
def test_power_cube_tets(gpu, n, seed, spread, brute):
    """The unit cube as 6 tetrahedra: weights in the paper's range +-|M|/n, and a
    spread that leaves dominated sites with empty cells."""
    w = I.workload("cube", n=n, seed=I.SEED_BASE + seed)
    d, r, err = _check(w, _weights(n, 1.0, seed, spread), brute=brute)
    if spread > 1:
        assert (r["measure"] == 0).any()
    print("cube", n, spread, err)
    d.close()


def test_power_lattice_mesh(gpu):
    """A 3x3x3 Kuhn lattice (162 tetrahedra): pieces cross many simplex faces."""
    v, s = I.kuhn_lattice_tets(3)
    n = 2500
    w = dict(name="pl", mode=B.MODE_3D, sites=I.uniform_sites(n, 3, I.SEED_BASE + 64), verts=v, simp=s, f64=False)
    d, r, err = _check(w, _weights(n, 1.0, 64))
    d.close()


def test_power_shell_clusters(gpu):
    """A small tetrahedralised shell with clustered sites (non-convex domain)."""
    v, s = I.small_shell(8)
    n = 3000
    w = dict(name="ps", mode=B.MODE_3D, sites=I.shell_sites(n, seed=I.SEED_BASE + 65, ncomp=4), verts=v, simp=s,
             f64=False)
    d, r, err = _check(w, _weights(n, I.domain_measure(4, v, s), 65))
    d.close()


@pytest.mark.parametrize("n,seed", [(1500, 66), (6000, 67)])
def test_power_torus_surface(gpu, n, seed):
    """Restricted power diagram on a torus: sites on (and 1e-4 off) the surface."""
    v, s = I.small_torus(60, 20)
    w = dict(name="pt", mode=B.MODE_SURFACE, sites=I.surface_sites(n, v, s, I.SEED_BASE + seed), verts=v, simp=s,
             f64=False)
    d, r, err = _check(w, _weights(n, I.domain_measure(3, v, s), seed))
    print("torus", n, err)
    d.close()


def test_power_box_form(gpu):
    """The box form (one piece per site, clipped from the whole box)."""
    w = I.workload("box", n=4000, seed=I.SEED_BASE + 68)
    d, r, err = _check(w, _weights(4000, 1.0, 68), box=True)
    d.close()


def test_power_equal_weights_and_clearing(gpu):
    """Equal weights give the Voronoi diagram; clearing the weights returns to it."""
    w = I.workload("cube", n=4000, seed=I.SEED_BASE + 69)
    d = B.diagram_from_workload(w)
    vor = d.compute()
    d.set_weights(torch.full((4000,), 0.01, device="cuda"))
    pw = d.compute()
    assert torch.equal(vor["nbr_off"], pw["nbr_off"]) and torch.equal(vor["nbr_idx"], pw["nbr_idx"])
    rel = (pw["measure"].double() - vor["measure"].double()).abs() / vor["measure"].double()
    assert float(rel.max()) < 2e-5
    d.set_weights(None)
    again = d.compute()
    for k in KEYS:
        assert torch.equal(vor[k], again[k]), k
    d.close()


def test_power_ignores_lists_and_split(gpu):
    """With weights set, the learned form and the split fall back to the plain
    per-tetrahedron search: the same bytes as the plain options."""
    w = I.workload("cube", n=3000, seed=I.SEED_BASE + 70)
    d = B.diagram_from_workload(w)
    d.set_weights(torch.tensor(_weights(3000, 1.0, 70), device="cuda"))
    plain = d.compute()
    d.set_options(learned=1, topk=16, split=1, mapping=0)
    other = d.compute()
    for k in KEYS:
        assert torch.equal(plain[k], other[k]), k
    d.close()


def test_power_rejects_bad_weights(gpu):
    w = I.workload("cube", n=100, seed=I.SEED_BASE + 71)
    d = B.diagram_from_workload(w)
    bad = torch.zeros(100, device="cuda")
    bad[5] = float("inf")
    with pytest.raises(B.VDError) as e:
        d.set_weights(bad)
    assert e.value.code == -1
    d.close()
