"""Comparison of the CUDA path against the oracle (test helper)."""
import numpy as np
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B

MEAS_RTOL = 1e-5   # per-site measure, relative (the benchmark spec)
CENT_RTOL = 1e-5   # centroid: |dc| <= 1e-5 |c|


def gpu_run(w, options=None, candidates=None):
    d = B.diagram_from_workload(w, options=options)
    if candidates is not None:
        d.set_candidates(candidates)
    r = d.compute()
    p = d.pieces()
    return d, r, p


def gpu_topology(p):
    meas = p["measure"].cpu().numpy()
    a = p["simplex"].cpu().numpy()
    i = p["site"].cpu().numpy()
    off = p["flag_off"].cpu().numpy()
    fl = p["flags"].cpu().numpy()
    out = {}
    for q in np.nonzero(meas > 0)[0]:
        out[(int(a[q]), int(i[q]))] = tuple(sorted(int(x) for x in fl[off[q]:off[q + 1]]))
    return out


def gpu_csr(r):
    off = r["nbr_off"].cpu().numpy()
    idx = r["nbr_idx"].cpu().numpy()
    return [list(map(int, idx[off[i]:off[i + 1]])) for i in range(len(off) - 1)]


def whole_cell_topology(ot, gt, m):
    """The oracle's per-simplex topology with the pieces of every site that the GPU
    computed as one whole cell (piece (m, i), the split of Alg. 5) merged into
    (m, i): the union of their bisector flags.  Such a cell must lie inside the
    domain: none of its oracle pieces has a face on the domain boundary."""
    whole = {i for (a, i) in gt if a == m}
    out = {}
    for (a, i), fl in ot.items():
        if i in whole:
            assert O.FLAG_BOUNDARY not in fl, f"site {i} computed whole but its cell meets the boundary"
            out.setdefault((m, i), set()).update(f for f in fl if f >= 0)
        else:
            out[(a, i)] = fl
    return {k: tuple(sorted(v)) if isinstance(v, set) else v for k, v in out.items()}


def compare_full(w, r, p, oracle_pieces, sites_subset=None, meas_floor=0.0, split=False):
    """Bit-exact topology and neighbours; measures / centroids within tolerance.

    meas_floor > 0: measures are compared relative to max(m, meas_floor) (cells
    reaching into the domain from far away are computed in the frame of their
    site, whose FP32 error scales with the distance, not with the piece).
    split: whole-cell pieces (m, i) stand for all of the site's oracle pieces."""
    n = len(w["sites"])
    om, oc, onb = O.per_site(n, w["sites"], oracle_pieces)
    gm = r["measure"].double().cpu().numpy()
    gc = r["centroid"].double().cpu().numpy()
    gnb = gpu_csr(r)
    ids = np.arange(n) if sites_subset is None else np.asarray(sites_subset)
    ot = oracle_pieces.topology()
    gt = gpu_topology(p)
    if split:
        ot = whole_cell_topology(ot, gt, len(w["simp"]))
    if sites_subset is not None:
        s = set(int(x) for x in ids)
        gt = {k: v for k, v in gt.items() if k[1] in s}
        ot = {k: v for k, v in ot.items() if k[1] in s}
    missing = set(ot) - set(gt)
    extra = set(gt) - set(ot)
    assert not missing and not extra, f"pair sets differ: missing {sorted(missing)[:5]} extra {sorted(extra)[:5]}"
    bad = [k for k in ot if ot[k] != gt[k]]
    assert not bad, f"flag sets differ for {len(bad)} pieces, e.g. {bad[0]}: {ot[bad[0]]} vs {gt[bad[0]]}"
    for i in ids:
        assert gnb[i] == onb[i], f"neighbours of site {i}: {gnb[i]} vs {onb[i]}"
    rel = np.abs(gm[ids] - om[ids]) / np.maximum(om[ids], max(meas_floor, 1e-300))
    assert ((om[ids] == 0) == (gm[ids] == 0)).all()
    nz = om[ids] > 0
    assert rel[nz].max(initial=0) <= MEAS_RTOL, f"measure rel err {rel[nz].max()}"
    dc = np.linalg.norm(gc[ids] - oc[ids], axis=1)
    cn = np.linalg.norm(oc[ids], axis=1)
    if meas_floor > 0:  # centroid error of a piece grows as its measure shrinks below the floor
        cn = cn * np.maximum(1.0, meas_floor / np.maximum(om[ids], 1e-300))
    assert (dc <= CENT_RTOL * np.maximum(cn, 1e-30)).all(), f"centroid err {(dc / cn).max()}"
    return dict(max_meas_rel=float(rel[nz].max(initial=0)), max_cent_rel=float((dc / np.maximum(cn, 1e-30)).max()))
