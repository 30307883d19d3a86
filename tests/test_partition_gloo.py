"""Host logic of the partitioned diagram (paper_2509_07175_b300/parallel.py) on
CPU: Morton-range ownership, the merge of per-rank results, and the pair
exchange over torch.distributed with two and three gloo ranks.  The ranks drive
a stand-in for the library context that floods a fixed pair graph: each rank
clips only its own sites' pairs, sends the others' through its outbox, and the
loop must end with every reachable pair clipped once, by its owner."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2509_07175_b300 import parallel as P  # noqa: E402


def _key(a, i):
    return (a << 32) | i


class FakeDiagram:
    """Pairs (a, i) of a small graph: pair (a, i) leads to (a, i + 1) and to
    (a + 1, i) (positive and negative flags of a piece).  Seeds: (0, i) for every
    owned site i."""

    def __init__(self, n, m, owner, rank):
        self.n, self.m, self.owner, self.rank = n, m, owner, rank
        self.seen, self.clipped, self.out = set(), [], []

    def _push(self, k):
        if k in self.seen:
            return
        self.seen.add(k)
        if int(self.owner[k & 0xFFFFFFFF]) == self.rank:
            self.queue.append(k)
        else:
            self.out.append(k)

    def _flood(self):
        while self.queue:
            k = self.queue.pop()
            self.clipped.append(k)
            a, i = k >> 32, k & 0xFFFFFFFF
            if i + 1 < self.n:
                self._push(_key(a, i + 1))
            if a + 1 < self.m:
                self._push(_key(a + 1, i))

    def compute(self):
        self.queue, self.out = [], []
        for i in range(self.n):
            if int(self.owner[i]) == self.rank:
                self._push(_key(0, i))
        self._flood()
        return {"status": 0}

    def outbox(self):
        return torch.tensor(sorted(self.out), dtype=torch.int64)

    def resume(self, keys):
        self.out = []
        self.queue = []
        added = 0
        for k in keys.tolist():
            if k not in self.seen:
                added += 1
            self._push(k)
        self._flood()
        return {"status": 0}, added


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    from paper_2509_07175_b300 import parallel as PP

    dist.init_process_group("gloo", rank=rank, world_size=world)
    maxes, sums = bench.reduce_over_ranks(dist, [100.0 + 10 * rank], [7 + rank], "cpu")
    n, m = 40, 5
    owner = torch.tensor(PP.morton_owner(np.random.default_rng(3).random((n, 3)), world))
    ex = PP.DistExchange(dist, rank, world, "cpu")
    # the exchange alone: every rank sends the keys of sites 0..n-1 of simplex rank
    keys = torch.tensor([_key(rank, i) for i in range(n)], dtype=torch.int64)
    got, total = ex.exchange(keys, owner)
    # the whole loop on the stand-in context
    fd = FakeDiagram(n, m, owner, rank)
    _r, rounds = PP.compute(fd, owner, ex)
    # the moved sites of a partitioned Lloyd step: each rank's own rows, summed
    full = torch.arange(3 * n, dtype=torch.float32).view(n, 3) * 0.5
    part = torch.where((owner == rank)[:, None], full, torch.zeros_like(full))
    assembled = torch.equal(ex.sum_(part), full)
    q.put((rank, maxes, sums, sorted(got.tolist()), total, sorted(fd.clipped), rounds, assembled))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_and_flood(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    n, m = 40, 5
    owner = P.morton_owner(np.random.default_rng(3).random((n, 3)), world)
    # every rank sees the slowest rank's time and the summed counts
    for _, maxes, sums, *_rest in out:
        assert maxes == [100.0 + 10 * (world - 1)]
        assert sums == [sum(7 + r for r in range(world))]
    everything = set()
    for rank, _m, _s, got, total, clipped, rounds, assembled in out:
        assert assembled
        assert total == world * n
        want = sorted(_key(a, i) for a in range(world) for i in range(n) if owner[i] == rank)
        assert got == want
        assert all(owner[k & 0xFFFFFFFF] == rank for k in clipped)  # only its own sites' pairs
        assert len(set(clipped)) == len(clipped)                     # each at most once
        everything |= set(clipped)
        assert rounds >= 1
    # together: every pair of the graph, exactly once over all ranks
    assert everything == {_key(a, i) for a in range(m) for i in range(n)}
    assert sum(len(c[5]) for c in out) == m * n


def test_morton_owner_ranges():
    rng = np.random.default_rng(7)
    s = rng.random((1001, 3))
    for world in (1, 2, 3, 8):
        o = P.morton_owner(s, world)
        cnt = np.bincount(o, minlength=world)
        assert cnt.max() - cnt.min() <= 1 and cnt.sum() == len(s)
        # contiguous in Morton order: the owner never decreases along the code order
        order = np.lexsort((np.arange(len(s)), P.morton_codes(s)))
        assert (np.diff(o[order]) >= 0).all()
    # Morton code of a point: bits of x, y, z interleaved (x lowest)
    c = P.morton_codes(np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.5, 0.0, 0.0], [0.0, 0.5, 0.0]]))
    assert c[0] == 0 and c[1] == (1 << 30) - 1
    assert c[2] == 1 << 27 and c[3] == 1 << 28


def test_local_exchange_and_merge():
    n = 6
    owner = torch.tensor([0, 1, 1, 0, 2, 2])
    ex = P.LocalExchange(3)
    outs = [torch.tensor([_key(3, 1), _key(4, 4)]), torch.tensor([_key(1, 0)]), torch.zeros(0, dtype=torch.int64)]
    inbox, total = ex.route(outs, owner)
    assert total == 3
    assert inbox[0].tolist() == [_key(1, 0)] and inbox[1].tolist() == [_key(3, 1)] and inbox[2].tolist() == [_key(4, 4)]
    # merge: each rank final for its own sites, zeros / empty lists elsewhere
    res = []
    for r in range(3):
        mine = owner == r
        meas = torch.where(mine, torch.arange(n, dtype=torch.float32) + 1, torch.zeros(n))
        cen = torch.where(mine[:, None], torch.arange(3 * n, dtype=torch.float32).view(n, 3), torch.zeros(n, 3))
        lists = [[i + 10, i + 20] if mine[i] else [] for i in range(n)]
        off = torch.tensor(np.concatenate([[0], np.cumsum([len(x) for x in lists])]), dtype=torch.int64)
        idx = torch.tensor([j for x in lists for j in x], dtype=torch.int32)
        res.append({"measure": meas, "centroid": cen, "nbr_off": off, "nbr_idx": idx})
    mg = P.merge(res, owner)
    assert torch.equal(mg["measure"], torch.arange(n, dtype=torch.float32) + 1)
    assert torch.equal(mg["centroid"], torch.arange(3 * n, dtype=torch.float32).view(n, 3))
    assert mg["nbr_off"].tolist() == [0, 2, 4, 6, 8, 10, 12]
    assert mg["nbr_idx"].tolist() == [j for i in range(n) for j in (i + 10, i + 20)]


def test_single_process_reduction_and_rate():
    import bench
    assert bench.reduce_over_ranks(None, [3.0], [4], "cpu") == ([3.0], [4])
    assert bench.whole_job_rate(1000, 10, 2000.0) == 5000.0
