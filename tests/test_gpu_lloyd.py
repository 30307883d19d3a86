"""Lloyd's method (Sec. 6.4, unit density) through vd_lloyd, with and without a
CUDA graph, against the oracle at every iteration.

Each iteration computes the diagram of the current sites and moves every site
with a non-empty cell to its cell's centroid.  Parity is per iteration: the
oracle recomputes the diagram from the GPU's own iterate (FP32 and FP64
trajectories are not compared with each other, they may drift apart).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_full, compare_population

pytestmark = pytest.mark.gpu


def _diag(w, **opt):
    return B.diagram_from_workload(w, options=opt or None)


def _result(d):
    """The diagram of the last iteration, read through vd_copy_result_host."""
    n, dt = d.n, d.dtype
    meas = torch.empty(n, dtype=dt)
    cen = torch.empty((n, 3), dtype=dt)
    off = torch.empty(n + 1, dtype=torch.int64)
    d.copy_result_host(meas, cen, off, None)
    nnz = int(off[-1])
    idx = torch.empty(max(nnz, 1), dtype=torch.int32)
    d.copy_result_host(meas, cen, off, idx)
    return {"measure": meas, "centroid": cen, "nbr_off": off, "nbr_idx": idx[:nnz].clone()}


def _sites_np(d, w):
    s = d.sites().double().cpu().numpy()
    if w["mode"] == B.MODE_2D:
        s[:, 2] = 0.0
    return s


@pytest.mark.parametrize("name,n,iters", [("cube", 100_000, 10), ("square", 1000, 10)])
def test_graph_equals_eager(gpu, name, n, iters):
    w = I.workload(name, n=n)
    a, b = _diag(w), _diag(w)
    a.lloyd(iters, use_graph=True)
    b.lloyd(iters, use_graph=False)
    assert torch.equal(a.sites(), b.sites())
    ra, rb = _result(a), _result(b)
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k
    a.close()
    b.close()


def test_cube_10_iterations_graph_per_iteration_parity(gpu):
    """Config 2: 100,000 uniform sites in the 6-tet cube, 10 Lloyd iterations
    replayed from one captured graph; at every iteration the diagram of that
    iteration's sites matches the oracle on every site, the update moves each
    site exactly to its centroid, and the mean displacement shrinks."""
    w = I.workload("cube")
    d = _diag(w)
    moves = []
    for it in range(10):
        s_before = _sites_np(d, w)
        d.lloyd(1, use_graph=True)
        r = _result(d)
        s_after = _sites_np(d, w)
        m = r["measure"].double().numpy()
        c = r["centroid"].double().numpy()
        assert (m > 0).all()
        assert np.array_equal(s_after, c)   # v_i <- centroid_i, bit for bit
        moves.append(float(np.linalg.norm(s_after - s_before, axis=1).mean()))
        wk = dict(w, sites=s_before)
        op = O.Oracle(4, s_before, w["verts"], w["simp"]).all_sites()
        compare_population(wk, r, d.pieces(), op)
    assert all(moves[k + 1] < moves[k] for k in range(len(moves) - 1)), moves
    d.close()


def test_torus_50_iterations_graph(gpu):
    """Config 4: restricted diagram on the 500,000-triangle torus, 200,000
    sites, 50 graph-captured Lloyd iterations; the 50th iteration's diagram
    matches the oracle on every site and partitions the surface."""
    w = I.workload("torus")
    d = _diag(w, stats=1)
    d.lloyd(49, use_graph=True)
    s49 = _sites_np(d, w)
    d.lloyd(1, use_graph=True)
    r = _result(d)
    p = d.pieces()
    pm = p["measure"].double().cpu().numpy()
    total = I.domain_measure(w["mode"], w["verts"], w["simp"])
    assert abs(pm.sum() - total) < 1e-5 * total
    op = O.Oracle(w["mode"], s49, w["verts"], w["simp"]).all_sites()
    compare_population(dict(w, sites=s49), r, p, op)
    d.close()


def test_learned_lloyd_trajectory_equals_plain(gpu):
    """The learned form with the network's ranking, captured in the graph, gives
    the same Lloyd trajectory bit for bit as the plain search."""
    w = I.workload("cube", n=30_000)
    a, b = _diag(w), _diag(w)
    b.mlp_init(11)
    b.set_options(learned=1, proposal=B.PROPOSAL_MLP, topk=16)
    a.lloyd(5, use_graph=True)
    b.lloyd(5, use_graph=True)
    assert torch.equal(a.sites(), b.sites())
    a.close()
    b.close()


def test_lloyd_zero_iterations_and_errors(gpu):
    w = I.workload("cube", n=1000)
    d = _diag(w)
    s0 = d.sites()
    d.lloyd(0)
    assert torch.equal(s0, d.sites())
    with pytest.raises(B.VDError):
        d.lloyd(-1)
    d.close()
