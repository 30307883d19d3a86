"""One diagram partitioned across ranks by site ownership (vd_set_partition,
vd_get_outbox, vd_resume; paper_2509_07175_b300/parallel.py).  The ranks run as
contexts one after the other on this GPU (no kernel of one waits on another's)
and exchange their outboxes on the host; the merged per-site result must equal
the one-context result bit for bit, every rank clips only its own sites'
pairs, and every pair is clipped by exactly one rank."""
import numpy as np
import pytest
import torch

from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I
from paper_2509_07175_b300 import parallel as P

pytestmark = pytest.mark.gpu

KEYS = ("measure", "centroid", "nbr_off", "nbr_idx")

CASES = [
    ("cube", 20000, dict(mapping=1)),
    ("cube", 20000, dict(learned=1, topk=16, mapping=1)),
    ("cube", 20000, dict(mapping=2)),                                  # thread per pair
    ("cube2m", 200000, dict(learned=1, topk=24, split=1, mapping=1)),
    ("shell", 30000, dict(learned=1, topk=24, mapping=1)),
    ("shell", 30000, dict(learned=1, topk=24, split=1, mapping=1)),
    ("box", 3000, dict(mapping=1)),
    ("torus", 20000, dict(learned=1, topk=16, mapping=1)),
    ("square", 1000, dict(mapping=1)),
]


def _ranks(w, opts, world):
    owner = torch.tensor(P.morton_owner(w["sites"], world), device="cuda")
    ds = []
    for r in range(world):
        d = B.diagram_from_workload(w, options=opts)
        d.set_partition(owner, r)
        ds.append(d)
    return ds, owner


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name,n,opts", CASES)
def test_partition_equals_one_context(gpu, name, n, opts, world):
    w = I.workload(name, n=n)
    one = B.diagram_from_workload(w, options=opts)
    full = one.compute()
    pairs_full = full["stats"]["pairs"]
    one.close()
    ds, owner = _ranks(w, dict(opts, stats=1), world)
    rs, rounds = P.compute_local(ds, owner)
    merged = P.merge(rs, owner)
    for k in KEYS:
        assert torch.equal(merged[k], full[k]), (name, k)
    own = owner.cpu().numpy()
    total = 0
    for r, d in enumerate(ds):
        p = d.pieces()
        sites = p["site"].cpu().numpy()
        assert (own[sites] == r).all()
        total += int(rs[r]["stats"]["pairs"])
        assert d.outbox().numel() == 0  # settled
    # each pair clipped once, by its owner (the one-context pair set, split among the ranks)
    assert total == pairs_full
    if opts.get("split") or name == "box":
        assert rounds == 0  # negative flags only, or no flood: nothing to exchange
    print(name, opts, "world", world, "rounds", rounds)
    for d in ds:
        d.close()


def test_partition_power_diagram(gpu):
    """A power diagram (3D, lifted sites) partitioned over two ranks."""
    w = I.workload("cube", n=5000)
    wt = torch.tensor(np.random.default_rng(5).uniform(-1, 1, len(w["sites"])) * 1e-5,
                      dtype=torch.float32, device="cuda")
    one = B.diagram_from_workload(w, options=dict(mapping=1))
    one.set_weights(wt)
    full = one.compute()
    one.close()
    ds, owner = _ranks(w, dict(mapping=1), 2)
    for d in ds:
        d.set_weights(wt)
    rs, _ = P.compute_local(ds, owner)
    merged = P.merge(rs, owner)
    for k in KEYS:
        assert torch.equal(merged[k], full[k]), k


def test_resume_rejects_bad_keys_and_lloyd(gpu):
    w = I.workload("cube", n=2000)
    ds, owner = _ranks(w, dict(mapping=1), 2)
    ds[0].compute()
    for bad in ((1 << 32) | 5000,              # a site index past n
                (len(w["simp"]) << 32) | 7):   # the whole-cell index m without the split
        ds[0].compute()
        with pytest.raises(B.VDError) as e:
            ds[0].resume(torch.tensor([bad], dtype=torch.int64, device="cuda"))
        assert e.value.code == -1
    with pytest.raises(B.VDError) as e:  # the partitioned context cannot run Lloyd alone
        ds[1].lloyd(1)
    assert e.value.code == -8
    # without a partition the outbox stays empty and resume with no keys is a no-op
    ds[1].set_partition(None, 0)
    r0 = ds[1].compute()
    assert ds[1].outbox().numel() == 0
    r1, added = ds[1].resume(torch.zeros(0, dtype=torch.int64, device="cuda"))
    assert added == 0
    for k in KEYS:
        assert torch.equal(r0[k], r1[k]), k
    for d in ds:
        d.close()


@pytest.mark.parametrize("name,n,opts", [("cube", 5000, dict(mapping=1)),
                                         ("shell", 20000, dict(learned=1, topk=24, split=1, mapping=1))])
def test_partitioned_lloyd(gpu, name, n, opts):
    """Lloyd iterations (Sec. 6.4) over two ranks: each rank moves its own sites
    (vd_lloyd_step) and the moved sites are assembled from their owners; the
    trajectory equals one context's vd_lloyd bit for bit."""
    w = I.workload(name, n=n)
    one = B.diagram_from_workload(w, options=opts)
    one.lloyd(3, use_graph=False)
    want = one.sites()
    one.close()
    ds, owner = _ranks(w, opts, 2)
    P.lloyd_local(ds, owner, 3)
    for d in ds:
        assert torch.equal(d.sites(), want)
        d.close()


@pytest.mark.parametrize("n", [1, 3])
def test_more_ranks_than_sites(gpu, n):
    """Four ranks over one or three sites: ranks that own nothing seed nothing
    and still take part in the exchange; the merged result is the one-context one."""
    w = I.workload("cube", n=n, seed=I.SEED_BASE + 0x3A0 + n)
    one = B.diagram_from_workload(w, options=dict(mapping=1))
    full = one.compute()
    one.close()
    ds, owner = _ranks(w, dict(mapping=1), 4)
    rs, _ = P.compute_local(ds, owner)
    merged = P.merge(rs, owner)
    for k in KEYS:
        assert torch.equal(merged[k], full[k]), k
    for d in ds:
        d.close()
