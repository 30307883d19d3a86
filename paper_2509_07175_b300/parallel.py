"""Partition of one diagram across ranks (host orchestration, argument routing only).

The pieces P_{a,i} are independent (Sec. 4: the GPU method needs no
synchronisation between pairs), so one diagram splits across ranks by site
ownership: sites are owned by contiguous ranges of their Morton order (equal
counts), every rank holds all sites and the whole domain (nearest-site queries
need them), and each rank computes the pieces of the sites it owns
(``vd_set_partition``).  A pair (T, j) that a rank's flood finds for a site j
of another rank (a positive flag, Alg. 4) leaves through the rank's outbox; the
exchange delivers it to j's owner, whose ``vd_resume`` clips it and floods on,
until no rank has outgoing pairs.  The split form (Alg. 5) floods through
negative flags only, so its outboxes stay empty and the exchange is one
count.  Per Lloyd iteration the moved sites are assembled from their owners.

Two exchanges route the outboxes: ``DistExchange.exchange(keys, owner) ->
(received, total)`` over ``torch.distributed`` (one rank per GPU; gathers of
counts and keys, which every backend provides) and ``LocalExchange``, which
emulates the ranks inside one process by running their contexts one after the
other (no kernel of one waits on another's).  The device work stays in libvd.
"""
from __future__ import annotations

import numpy as np
import torch

KEY_SITE_MASK = 0xFFFFFFFF


def morton_codes(sites) -> np.ndarray:
    """30-bit Morton codes of the sites over their bounding box (10 bits per axis)."""
    s = np.asarray(sites, dtype=np.float64)
    lo, hi = s.min(axis=0), s.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    q = np.clip(((s - lo) / span * 1024.0).astype(np.int64), 0, 1023)

    def spread(v):  # 10 bits -> every third bit
        v = (v | (v << 16)) & 0x030000FF
        v = (v | (v << 8)) & 0x0300F00F
        v = (v | (v << 4)) & 0x030C30C3
        v = (v | (v << 2)) & 0x09249249
        return v

    code = spread(q[:, 0]) | (spread(q[:, 1]) << 1)
    if s.shape[1] > 2:
        code |= spread(q[:, 2]) << 2
    return code


def morton_owner(sites, world: int) -> np.ndarray:
    """Owner rank of each site: equal-count contiguous ranges of the Morton order
    (ties in the code broken by site index)."""
    n = len(sites)
    order = np.lexsort((np.arange(n), morton_codes(sites)))
    owner = np.empty(n, dtype=np.int32)
    owner[order] = (np.arange(n, dtype=np.int64) * world // max(n, 1)).astype(np.int32)
    return owner


def destinations(keys: torch.Tensor, owner: torch.Tensor) -> torch.Tensor:
    """Owner rank of each pair key (simplex << 32) | site."""
    return owner[(keys & KEY_SITE_MASK).long()].long()


class LocalExchange:
    """All ranks in one process: each rank's outbox is held until every rank has
    posted, then routed."""

    def __init__(self, world: int):
        self.world = world

    def route(self, outs, owner):
        """outs[r]: keys of rank r -> (inbox per rank, total keys sent)."""
        inbox = [[] for _ in range(self.world)]
        total = 0
        for keys in outs:
            total += int(keys.numel())
            if keys.numel() == 0:
                continue
            dest = destinations(keys, owner)
            for r in range(self.world):
                sel = keys[dest == r]
                if sel.numel():
                    inbox[r].append(sel)
        dev = owner.device
        return [torch.cat(b) if b else torch.zeros(0, dtype=torch.int64, device=dev) for b in inbox], total


class DistExchange:
    """One rank per process over torch.distributed: counts and keys are gathered
    from every rank (padded to the largest outbox) and each rank keeps the keys
    its sites own.  Works with the nccl backend on CUDA tensors and with gloo on
    CPU tensors."""

    def __init__(self, dist, rank: int, world: int, device="cuda"):
        self.dist, self.rank, self.world, self.device = dist, rank, world, torch.device(device)

    def exchange(self, keys: torch.Tensor, owner: torch.Tensor):
        keys = keys.to(self.device, torch.int64)
        cnt = torch.tensor([keys.numel()], dtype=torch.int64, device=self.device)
        counts = [torch.zeros_like(cnt) for _ in range(self.world)]
        self.dist.all_gather(counts, cnt)
        counts = [int(c.item()) for c in counts]
        total = sum(counts)
        if total == 0:
            return torch.zeros(0, dtype=torch.int64, device=self.device), 0
        width = max(counts)
        pad = torch.full((width,), -1, dtype=torch.int64, device=self.device)
        pad[:keys.numel()] = keys
        got = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(got, pad)
        allk = torch.cat([g[:c] for g, c in zip(got, counts)])
        mine = allk[destinations(allk, owner.to(self.device)) == self.rank]
        return mine, total

    def sum_(self, t: torch.Tensor) -> torch.Tensor:
        x = t.to(self.device)
        self.dist.all_reduce(x)
        return x


def compute(d, owner: torch.Tensor, ex: DistExchange, max_rounds: int = 64):
    """One partitioned computation on this rank: vd_compute, then rounds of
    outbox exchange and vd_resume until no rank sends a pair.  Returns the rank's
    result (final for its own sites) and the number of exchange rounds."""
    r = d.compute()
    rounds = 0
    while True:
        recv, total = ex.exchange(d.outbox(), owner)
        if total == 0:
            return r, rounds
        if rounds == max_rounds:
            raise RuntimeError(f"pair exchange did not settle in {max_rounds} rounds")
        r, _ = d.resume(recv)
        rounds += 1


def compute_local(diagrams, owner: torch.Tensor, max_rounds: int = 64):
    """The same with every rank's context in this process (LocalExchange)."""
    ex = LocalExchange(len(diagrams))
    rs = [d.compute() for d in diagrams]
    rounds = 0
    while True:
        inbox, total = ex.route([d.outbox() for d in diagrams], owner)
        if total == 0:
            return rs, rounds
        if rounds == max_rounds:
            raise RuntimeError(f"pair exchange did not settle in {max_rounds} rounds")
        for k, d in enumerate(diagrams):
            rs[k], _ = d.resume(inbox[k])
        rounds += 1


def merge(results, owner: torch.Tensor):
    """Assemble the per-site outputs of all ranks (each final for the sites it
    owns): measure, centroid and the neighbour CSR, as one diagram's."""
    n = owner.numel()
    dev = results[0]["measure"].device
    own = owner.to(dev).long()
    ar = torch.arange(n, device=dev)
    measure = torch.stack([r["measure"] for r in results])[own, ar]
    centroid = torch.stack([r["centroid"] for r in results])[own, ar]
    cnts = torch.stack([r["nbr_off"][1:] - r["nbr_off"][:-1] for r in results])
    cnt = cnts[own, ar]
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(cnt, 0)
    idx = torch.empty(int(off[-1].item()), dtype=torch.int32, device=dev)
    for k, r in enumerate(results):
        sites = torch.nonzero(own == k).flatten()
        c = cnt[sites]
        tot = int(c.sum().item())
        if tot == 0:
            continue
        seg = torch.repeat_interleave(torch.arange(sites.numel(), device=dev), c)
        within = torch.arange(tot, device=dev) - torch.repeat_interleave(torch.cumsum(c, 0) - c, c)
        idx[off[sites][seg] + within] = r["nbr_idx"][r["nbr_off"][sites][seg] + within]
    return {"measure": measure, "centroid": centroid, "nbr_off": off, "nbr_idx": idx}


def _assemble_sites(moved, owner):
    """The sites as their owners moved them: rank r's copy supplies the rows it owns."""
    own = owner.to(moved[0].device).long()
    ar = torch.arange(own.numel(), device=own.device)
    return torch.stack(moved)[own, ar]


def lloyd_local(diagrams, owner: torch.Tensor, iters: int):
    """Lloyd iterations (Sec. 6.4) of a partitioned diagram whose ranks are
    contexts of this process: per iteration the partitioned compute, each rank's
    update of its own sites (vd_lloyd_step), and the moved sites assembled from
    their owners into every rank (vd_update_sites)."""
    rounds = []
    for _ in range(iters):
        _rs, rd = compute_local(diagrams, owner)
        rounds.append(rd)
        moved = []
        for d in diagrams:
            d.lloyd_step()
            moved.append(d.sites())
        sites = _assemble_sites(moved, owner)
        for d in diagrams:
            d.update_sites(sites[:, :d.dim])
    return rounds


def lloyd(d, owner: torch.Tensor, ex: DistExchange, iters: int):
    """The same with one rank per process: the moved sites travel in one
    all-reduce of the owners' rows (12 B per site per iteration in FP32)."""
    own = (owner.to("cuda") == ex.rank)
    rounds = []
    for _ in range(iters):
        _r, rd = compute(d, owner, ex)
        rounds.append(rd)
        d.lloyd_step()
        s = d.sites()
        part = torch.where(own[:, None], s, torch.zeros_like(s))
        d.update_sites(ex.sum_(part).to("cuda")[:, :d.dim])
    return rounds
