"""Power diagrams in the plane (the paper's lifting extension) against the oracle.

The library lifts each weighted site to (x, y, sqrt(eta - w)) and computes the
restricted diagram on the planar mesh; the oracle clips the triangles by power
bisectors directly, with the weights the lift realises exactly (-h^2 for the
float height h; a constant shift of all weights changes nothing)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I
from vdcheck import CENT_RTOL, MEAS_RTOL, gpu_csr, gpu_topology

pytestmark = pytest.mark.gpu


def _case(n, seed, grid=1, spread=1.0):
    if grid == 1:
        v, t = I.square_2tri()
    else:
        v, t = I.square_grid_tris(grid)  # dyadic grids: vertices exact in float32
    xy = I.uniform_sites(n, 2, seed)[:, :2]
    rng = np.random.default_rng(seed + 1)
    w = (rng.uniform(-1.0, 1.0, n) * spread / n).astype(np.float32).astype(np.float64)  # |M| = 1
    return v, t, xy, w


def _run(v, t, xy, w, **opt):
    d = B.Diagram(torch.tensor(xy, dtype=torch.float32, device="cuda"),
                  torch.tensor(v[:, :2], dtype=torch.float32, device="cuda"),
                  torch.tensor(t, dtype=torch.int32, device="cuda"),
                  weights=torch.tensor(w, dtype=torch.float32, device="cuda"), options=opt or None)
    r = d.compute()
    return d, r


def _check(v, t, xy, d, r, brute):
    lifted = d.sites().double().cpu().numpy()
    assert np.array_equal(lifted[:, :2], xy.astype(np.float32).astype(np.float64))
    om_w = -lifted[:, 2] ** 2            # the weights the float lift realises
    sites0 = np.c_[xy, np.zeros(len(xy))]
    op = O.Oracle(2, sites0, v, t, brute=brute, weights=om_w).enumerate()
    assert op.stats["uncertain"] == 0
    n = len(xy)
    om, oc, onb = O.per_site(n, sites0, op)
    gm = r["measure"].double().cpu().numpy()
    gc = r["centroid"].double().cpu().numpy()
    assert ((om > 0) == (gm > 0)).all()
    nz = om > 0
    # FP32 in the frame of the lifted site: a cell much smaller than the lift height
    # carries an error scaled by the typical cell, so the bound is 1e-5 of
    # max(m, |M| / n) (|M| = 1); neighbours and topology stay exact
    mbar = 1.0 / n
    err = np.abs(gm[nz] - om[nz]) / np.maximum(om[nz], mbar)
    assert err.max() <= MEAS_RTOL, err.max()
    dc = np.linalg.norm(gc[nz] - oc[nz], axis=1)
    assert (dc <= CENT_RTOL * np.linalg.norm(oc[nz], axis=1)).all()
    assert gpu_csr(r) == onb
    gt = gpu_topology(d.pieces())
    assert gt == op.topology()
    return int((~nz).sum())


@pytest.mark.parametrize("n,seed,grid,spread,brute", [(60, 3, 1, 1.0, True), (400, 5, 2, 1.0, True),
                                                      (3000, 7, 4, 1.0, False), (2000, 9, 2, 8.0, False)])
def test_power_against_oracle(gpu, n, seed, grid, spread, brute):
    v, t, xy, w = _case(n, seed, grid, spread)
    d, r = _run(v, t, xy, w)
    assert r["status"] == 0 and r["stats"]["uncertain"] == 0
    empty = _check(v, t, xy, d, r, brute)
    if spread > 1.0:
        assert empty > 0   # strong weights leave some sites without a cell
    assert abs(float(r["measure"].double().sum()) - 1.0) < 1e-5
    d.close()


def test_power_equal_weights_is_voronoi(gpu):
    v, t, xy, _ = _case(2000, 11, 4)
    d, r = _run(v, t, xy, np.full(len(xy), 0.25))
    w = dict(name="sq", mode=2, sites=np.c_[xy, np.zeros(len(xy))], verts=v, simp=t, f64=False)
    rv = B.diagram_from_workload(w).compute()
    assert torch.equal(r["nbr_off"], rv["nbr_off"]) and torch.equal(r["nbr_idx"], rv["nbr_idx"])
    rel = (r["measure"].double() - rv["measure"].double()).abs() / rv["measure"].double()
    assert float(rel.max()) < 2e-5
    d.close()


def test_power_learned_form_bitwise(gpu):
    v, t, xy, w = _case(20000, 13, 4)
    d, plain = _run(v, t, xy, w)
    d.set_options(learned=1, topk=16)
    lr = d.compute()
    for k in ("measure", "centroid", "nbr_off", "nbr_idx"):
        assert torch.equal(plain[k], lr[k]), k
    d.close()


def test_power_rejects_bad_weights(gpu):
    v, t, xy, w = _case(10, 15)
    w[3] = np.nan
    with pytest.raises(B.VDError) as e:
        _run(v, t, xy, w)
    assert e.value.code == -1
