"""The population checker used by the GPU parity tests, run on the CPU: fed the
oracle's own pieces in the layout the C ABI returns, it passes; with a mistake
planted in that stand-in (a dropped face flag, a dropped piece, a moved
neighbour, a measure off by more than the bar) it fails -- in the whole and in
the site-subset mode."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_07175_b300 import inputs as I
from vdcheck import compare_population


def _as_result(n, sites, op):
    """(r, p): the oracle's pieces in the layout of vd_get_pieces / vd_result."""
    keep = np.nonzero(op.meas > 0)[0]
    cnt = (op.foff[1:] - op.foff[:-1])[keep]
    foff = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    flags = np.concatenate([op.flags[op.foff[k]:op.foff[k + 1]] for k in keep]) if len(keep) else np.zeros(0, np.int32)
    p = dict(simplex=torch.tensor(op.a[keep].astype(np.int32)), site=torch.tensor(op.i[keep].astype(np.int32)),
             measure=torch.tensor(op.meas[keep].astype(np.float32)), flag_off=torch.tensor(foff),
             flags=torch.tensor(flags.astype(np.int32)))
    om, oc, onb = O.per_site(n, sites, op)
    off = np.concatenate([[0], np.cumsum([len(x) for x in onb])]).astype(np.int64)
    idx = np.array([j for x in onb for j in x], dtype=np.int32)
    r = dict(measure=torch.tensor(om.astype(np.float32)), centroid=torch.tensor(oc.astype(np.float32)),
             nbr_off=torch.tensor(off), nbr_idx=torch.tensor(idx))
    return r, p


@pytest.fixture(scope="module")
def case():
    v, s = I.kuhn_lattice_tets(3)
    sites = I.uniform_sites(1500, 3, I.SEED_BASE + 0x7A1)
    w = dict(mode=4, sites=sites, verts=v, simp=s)
    op = O.Oracle(4, sites, v, s).all_sites()
    return w, op


def _plant(r, p, what):
    r = {k: t.clone() for k, t in r.items()}
    p = {k: t.clone() for k, t in p.items()}
    if what == "flag":       # one bisector flag of one piece replaced by another site
        j = int(torch.nonzero(p["flags"] >= 0)[5])
        p["flags"][j] = (p["flags"][j] + 1) % len(r["measure"])
    elif what == "piece":    # one piece reported empty
        p["measure"][7] = 0.0
    elif what == "nbr":      # one neighbour id changed
        r["nbr_idx"][11] = (r["nbr_idx"][11] + 3) % len(r["measure"])
    elif what == "measure":  # one site's measure off by 3e-5 relative
        r["measure"][13] *= 1 + 3e-5
    return r, p


def test_checker_accepts_the_oracle(case):
    w, op = case
    r, p = _as_result(len(w["sites"]), w["sites"], op)
    out = compare_population(w, r, p, op)
    assert out["pieces"] == int((op.meas > 0).sum())


@pytest.mark.parametrize("what", ["flag", "piece", "nbr", "measure"])
def test_checker_catches_planted_mistakes(case, what):
    w, op = case
    r, p = _as_result(len(w["sites"]), w["sites"], op)
    r, p = _plant(r, p, what)
    with pytest.raises(AssertionError):
        compare_population(w, r, p, op)


def test_checker_site_subset(case):
    """ids mode: the result of every site against the oracle's pieces of a subset;
    a planted mistake at a subset site fails, one outside the subset is not seen."""
    w, op_all = case
    n = len(w["sites"])
    r, p = _as_result(n, w["sites"], op_all)
    ids = np.sort(np.random.default_rng(5).choice(n, 300, replace=False))
    op = O.Oracle(4, w["sites"], w["verts"], w["simp"]).site_pieces(ids)
    out = compare_population(w, r, p, op, ids=ids)
    assert out["sites"] == 300
    inside, outside = int(ids[4]), int(np.setdiff1d(np.arange(n), ids)[4])
    for site, fails in ((inside, True), (outside, False)):
        r2 = {k: t.clone() for k, t in r.items()}
        r2["measure"][site] *= 1 + 3e-5
        if fails:
            with pytest.raises(AssertionError):
                compare_population(w, r2, p, op, ids=ids)
        else:
            compare_population(w, r2, p, op, ids=ids)
    # a dropped flag of a piece of a subset site
    p2 = {k: t.clone() for k, t in p.items()}
    q = int(np.nonzero(np.isin(p["site"].numpy(), [inside]))[0][0])
    lo, hi = int(p["flag_off"][q]), int(p["flag_off"][q + 1])
    p2["flags"][lo:hi] = p2["flags"][lo]  # every flag of that piece the same value
    with pytest.raises(AssertionError):
        compare_population(w, r, p2, op, ids=ids)
