"""Comparison of the CUDA path against the oracle (test helper)."""
import numpy as np
import torch

import oracle as O
from paper_2509_07175_b300 import binding as B

MEAS_RTOL = 1e-5   # per-site measure, relative (the stated parity bar)
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


# ---------------------------------------------------------------------------
# whole-population comparison (vectorised: every site, every piece)
# ---------------------------------------------------------------------------
def _gather_flags(foff, flags, idx):
    """flags of pieces idx (in that order) as one array, with per-piece counts"""
    foff = np.asarray(foff, dtype=np.int64)
    cnt = (foff[1:] - foff[:-1])[idx]
    tot = int(cnt.sum())
    if tot == 0:
        return cnt, np.zeros(0, np.int64), np.zeros(0, np.int64)
    first = np.repeat(foff[idx] - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt)
    pos = first + np.arange(tot)
    owner = np.repeat(np.arange(len(idx)), cnt)
    return cnt, np.asarray(flags, dtype=np.int64)[pos], owner


def _pack(hi, lo):
    """one sortable int64 per (hi, lo) pair: hi >= 0 in the upper 32 bits, lo as a
    signed 32-bit value shifted to unsigned in the lower ones"""
    return (np.asarray(hi, np.int64) << 32) | (np.asarray(lo, np.int64) + 2 ** 31)


def _unpack(k):
    return k >> 32, (k & 0xFFFFFFFF) - 2 ** 31


def _unique_pairs(hi, lo):
    """sorted unique (hi, lo) rows, by a 1-D sort of packed keys"""
    if len(hi) == 0:
        return np.zeros((0, 2), np.int64)
    a, b = _unpack(np.unique(_pack(hi, lo)))
    return np.stack([a, b], 1)


def _canonical(keys, owner, fl, nkeys):
    """pieces sorted by key, each piece's flags sorted: (keys, counts, flags)"""
    order = np.argsort(keys, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    if len(fl):
        ro = rank[owner]
        _, fs = _unpack(np.sort(_pack(ro, fl)))
        cnt = np.bincount(ro, minlength=nkeys)
    else:
        fs, cnt = np.zeros(0, np.int64), np.zeros(nkeys, np.int64)
    return keys[order], cnt, fs


def _merge_sites(a, i, keep_idx, cnt, fl, owner, merged_sites, m_index, boundary_ok):
    """Pieces of the sites in merged_sites folded into one piece (m_index, i) whose
    flags are the union of their bisector flags (and FLAG_BOUNDARY once when
    boundary_ok and some piece of the site has it)."""
    site_of_piece = i[keep_idx]
    is_m = np.isin(site_of_piece, merged_sites)
    # the kept (unmerged) pieces
    k_idx = np.nonzero(~is_m)[0]
    k_mask = ~is_m[owner] if len(owner) else np.zeros(0, bool)
    k_keys = (a[keep_idx][k_idx].astype(np.int64) << 32) | site_of_piece[k_idx]
    remap = -np.ones(len(keep_idx), np.int64)
    remap[k_idx] = np.arange(len(k_idx))
    k_owner = remap[owner[k_mask]]
    k_fl = fl[k_mask]
    # merged: per site, unique flags >= 0, plus boundary
    m_mask = is_m[owner] if len(owner) else np.zeros(0, bool)
    ms = site_of_piece[owner[m_mask]]
    mf = fl[m_mask]
    bnd_sites = np.unique(ms[mf == FLAG_BOUNDARY_I64])
    sel = mf >= 0
    pairs = _unique_pairs(ms[sel], mf[sel])
    if boundary_ok and len(bnd_sites):
        pairs = np.concatenate([pairs, np.stack([bnd_sites, np.full(len(bnd_sites), FLAG_BOUNDARY_I64)], 1)])
    msites = np.unique(site_of_piece[is_m])
    m_keys = (np.int64(m_index) << 32) | msites
    mpos = np.searchsorted(msites, pairs[:, 0])
    keys = np.concatenate([k_keys, m_keys])
    owner2 = np.concatenate([k_owner, len(k_idx) + mpos])
    fl2 = np.concatenate([k_fl, pairs[:, 1]])
    return keys, owner2, fl2, bnd_sites


FLAG_BOUNDARY_I64 = np.int64(O.FLAG_BOUNDARY)


def compare_population(w, r, p, op, split=False, box=False, meas_floor=0.0, ids=None):
    """Every site and every piece of the CUDA result against the oracle (or, with
    ids -- sorted site indices -- every piece of those sites against the oracle's
    pieces of the same sites, op = site_pieces(ids)).

    Bit-exact: the set of non-empty pieces (simplex, site), each piece's sorted
    face flags, each site's neighbour list.  Within 1e-5: per-site measures
    (relative) and centroids (|dc| <= 1e-5 |c|).  split: the GPU's whole-cell
    pieces (m, i) stand for all of the site's oracle pieces (which must not touch
    the domain boundary); box: the GPU's one piece (0, i) per site stands for the
    site's pieces in the 6 tetrahedra of the box (boundary flag once if any).
    Returns the measured errors."""
    n = len(w["sites"])
    m = len(w["simp"])
    oa, oi = np.asarray(op.a, np.int64), np.asarray(op.i, np.int64)
    okeep = np.nonzero(op.meas > 0)[0]
    ocnt, ofl, oown = _gather_flags(op.foff, op.flags, okeep)
    ga = p["simplex"].cpu().numpy().astype(np.int64)
    gi = p["site"].cpu().numpy().astype(np.int64)
    gm = p["measure"].double().cpu().numpy()
    insub = np.ones(n, bool)
    if ids is not None:
        ids = np.asarray(ids, np.int64)
        assert (np.diff(ids) > 0).all()
        insub[:] = False
        insub[ids] = True
        assert insub[oi].all(), "oracle pieces outside the site subset"
    gkeep = np.nonzero((gm > 0) & insub[gi])[0]
    gcnt, gfl, gown = _gather_flags(p["flag_off"].cpu().numpy(), p["flags"].cpu().numpy(), gkeep)
    gkeys = (ga[gkeep] << 32) | gi[gkeep]
    if box and len(gfl):  # the box form flags each box face: the boundary counts once per site
        u = _unique_pairs(gown, gfl)
        gown, gfl = u[:, 0], u[:, 1]
    if split or box:
        merged = np.unique(gi[gkeep][ga[gkeep] == m]) if split else np.nonzero(insub)[0]
        okeys, oown2, ofl2, obnd = _merge_sites(oa, oi, okeep, ocnt, ofl, oown, merged, m if split else 0,
                                                boundary_ok=box)
        if split:
            assert len(obnd) == 0, f"sites computed whole touch the boundary: {obnd[:5]}"
        G = _canonical(gkeys, gown, gfl, len(gkeys))
        Ok = _canonical(okeys, oown2, ofl2, len(okeys))
    else:
        okeys = (oa[okeep] << 32) | oi[okeep]
        G = _canonical(gkeys, gown, gfl, len(gkeys))
        Ok = _canonical(okeys, oown, ofl, len(okeys))
    if not np.array_equal(G[0], Ok[0]):
        miss = np.setdiff1d(Ok[0], G[0])
        extra = np.setdiff1d(G[0], Ok[0])
        raise AssertionError(f"pair sets differ: {len(miss)} missing e.g. {[(int(k >> 32), int(k & 0xffffffff)) for k in miss[:3]]}, "
                             f"{len(extra)} extra e.g. {[(int(k >> 32), int(k & 0xffffffff)) for k in extra[:3]]}")
    if not (np.array_equal(G[1], Ok[1]) and np.array_equal(G[2], Ok[2])):
        bad = np.nonzero(G[1] != Ok[1])[0]
        if len(bad) == 0:  # same counts: the first piece whose flag values differ
            off = np.concatenate([[0], np.cumsum(G[1])])
            f = int(np.nonzero(G[2] != Ok[2])[0][0])
            bad = [int(np.searchsorted(off, f, side="right") - 1)]
        b = bad[0]
        raise AssertionError(f"flag sets differ for piece {(int(G[0][b] >> 32), int(G[0][b] & 0xffffffff))} "
                             f"({len(bad)} pieces)")
    # neighbours: unique positive flags per site over its pieces of positive measure
    sel = ofl >= 0
    pairs = _unique_pairs(oi[okeep][oown[sel]], ofl[sel])
    ocnt_site = np.bincount(pairs[:, 0], minlength=n)
    goff = r["nbr_off"].cpu().numpy().astype(np.int64)
    gidx = r["nbr_idx"].cpu().numpy().astype(np.int64)
    if ids is None:
        onoff = np.concatenate([[0], np.cumsum(ocnt_site)])
        assert np.array_equal(goff, onoff), "neighbour counts differ"
        assert np.array_equal(gidx, pairs[:, 1]), "neighbour lists differ"
    else:
        gcnt_site = goff[ids + 1] - goff[ids]
        assert np.array_equal(gcnt_site, ocnt_site[ids]), "neighbour counts differ"
        tot = int(gcnt_site.sum())
        first = np.repeat(goff[ids] - np.concatenate([[0], np.cumsum(gcnt_site)[:-1]]), gcnt_site)
        assert np.array_equal(gidx[first + np.arange(tot)], pairs[:, 1]), "neighbour lists differ"
    # per-site measure and centroid
    om = np.zeros(n)
    m1 = np.zeros((n, 3))
    np.add.at(om, oi[okeep], op.meas[okeep])
    np.add.at(m1, oi[okeep], op.m1[okeep])
    oc = np.asarray(w["sites"], dtype=np.float64).copy()
    ok = om > 0
    oc[ok] += m1[ok] / om[ok, None]
    gmm = r["measure"].double().cpu().numpy()
    gc = r["centroid"].double().cpu().numpy()
    if ids is not None:  # only the subset's rows
        om, oc, ok, gmm, gc = om[ids], oc[ids], ok[ids], gmm[ids], gc[ids]
        n = len(ids)
    assert ((gmm > 0) == ok).all(), "empty cells differ"
    # meas_floor > 0 (power diagrams): a cell far smaller than the lift height is
    # computed in the frame of its lifted site, so its error scales with the typical
    # cell: measures relative to max(m, floor), centroids likewise scaled
    rel = np.abs(gmm[ok] - om[ok]) / np.maximum(om[ok], meas_floor)
    dc = np.linalg.norm(gc - oc, axis=1)
    cn = np.linalg.norm(oc, axis=1)
    if meas_floor > 0:
        cn = cn * np.maximum(1.0, meas_floor / np.maximum(om, 1e-300))
    dim = 3 if w["mode"] == 4 else 2
    h = np.where(ok, np.maximum(om, 1e-300) ** (1.0 / dim), 1.0)
    out = dict(sites=int(n), pieces=int(len(G[0])), max_meas_rel=float(rel.max(initial=0)),
               max_cent_rel=float((dc / np.maximum(cn, 1e-30)).max(initial=0)),
               max_dc_over_h=float((dc[ok] / h[ok]).max(initial=0)))
    assert out["max_meas_rel"] <= MEAS_RTOL, out
    assert (dc <= CENT_RTOL * np.maximum(cn, 1e-30)).all(), out
    return out
