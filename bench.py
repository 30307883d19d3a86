#!/usr/bin/env python
"""Benchmark: clipped Voronoi cells per second on one B300 (or one diagram over N).

One step = one ``vd_compute`` through the C ABI: grid build, nearest-neighbour
distances, seeding, the persistent clip-and-flood kernel and the per-site
reduction (measure, centroid, neighbour CSR) for the whole workload.

value   device-resident inputs; per-step CUDA events on the compute stream;
        L2 flushed (256 MiB write) before every step, outside the events.
e2e     the same metric through the public API with host buffers: pinned host
        sites -> device, compute, results (measure, centroid, CSR) -> host.
roofline  the clip kernel (dominant), FP32-ALU bound: algorithmic FLOPs (8 per
        site-distance evaluation, counted by the library's counters) over its
        event-timed duration, against SMs x 128 lanes x 2 x max SM clock.
cpu_baseline  the FP64 CPU oracle on the whole workload (all host threads; one
        thread on a bounded sample), with the measured errors of the timed
        result against it (oracle_check) and the paper's serial method on one
        thread (serial_baseline).

Multi-GPU (torchrun): one diagram partitioned across the ranks by site
ownership (Morton ranges; paper_2509_07175_b300/parallel.py).  A step is the
partitioned compute with its pair exchange (gathers over NCCL until no rank
sends a pair); value = the workload's cells / max over ranks of the step time
(strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "shell"
METRIC = "clipped Voronoi cells/sec (3D, 1M sites) learned+batched vs plain GPU, oracle-exact"
UNIT = "cells/s"
DESC = {
    "cube": "3D clipped VD: unit cube as 6 tets, 100,000 uniform sites (FP32, FP64-filtered signs)",
    "cube1m": "3D clipped VD: unit cube as 6 tets, 1,000,000 uniform sites (FP32)",
    "shell": "3D clipped VD: tetrahedralised spherical shell (172,032 tets), 1,000,000 sites "
             "(16-component Gaussian mixture sigma 0.02 + 10% uniform), FP32",
    "cube2m": "3D clipped VD: unit cube as 6 tets, 2,000,000 uniform sites, FP32",
    "square": "2D clipped VD: unit square as 2 triangles, 1,000 uniform sites, FP64",
    "torus": "restricted VD: torus (500,000 triangles), 200,000 sites, FP32",
    "box": "3D clipped VD: unit cube as one convex domain (box form), 100,000 uniform sites, FP32",
    "box5m": "3D clipped VD: unit cube as one convex domain (box form), 5,000,000 uniform sites (white noise), FP32",
    "grid5m": "3D clipped VD: unit cube as one convex domain (box form), 171^3 = 5,000,211 sites on a "
              "perturbed grid (+-0.1 h), FP32",
    "blue5m": "3D clipped VD: unit cube as one convex domain (box form), 5,000,000 blue-noise sites: the "
              "white-noise sites relaxed by 100 graph-captured Lloyd iterations of this library (timed), FP32",
    "blue100k": "3D clipped VD: unit cube as one convex domain (box form), 100,000 Poisson-disk (blue noise) "
                "sites, FP32",
}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the 3D
# clip kernel, from a single-pass ncu capture of the learned form (top 24, split) on
# the full workload,
# valid only for the kernel sources it was taken on (their hash)
FLOOD_TRAFFIC = {"source_hash": "5a5f82d27e94b648",
                 "bytes": {"shell": 1.24e9 + 0.260e9}}


def _source_hash():
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2509_07175_b300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def flood_traffic(workload):
    """Captured bytes per launch, or None when the kernel changed since the capture."""
    if _source_hash() != FLOOD_TRAFFIC["source_hash"]:
        return None
    return FLOOD_TRAFFIC["bytes"].get(workload)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_over_ranks(dist, maxes, sums, device):
    """Element-wise MAX of `maxes` and SUM of `sums` over all ranks (no-op without
    a process group).  Used for the step time (max over ranks) and the counts."""
    if dist is None:
        return list(maxes), list(sums)
    import torch
    tm = torch.tensor(list(maxes), dtype=torch.float64, device=device)
    ts = torch.tensor(list(sums), dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return tm.tolist(), ts.tolist()


def whole_job_rate(units: int, steps: int, max_ms: float) -> float:
    """Units of the whole job (one diagram of `units` cells per step, however many
    ranks share it) per second of the slowest rank."""
    return units * steps / (max_ms / 1e3)


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(w, one_thread_s=8.0, seed=0):
    """The FP64 oracle on the host cores: the whole workload on all threads (its
    result also gives the bench line's measured errors), and a bounded sample of
    sites on one thread.  Returns (baseline dict, oracle pieces)."""
    import numpy as np

    import oracle as O

    cores = os.cpu_count() or 1
    n = len(w["sites"])
    o = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"], nthreads=cores)
    t0 = time.perf_counter()
    op = o.all_sites()
    dt = time.perf_counter() - t0
    o.close()
    o1 = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"], nthreads=1)
    rng = np.random.default_rng(seed)
    pilot = rng.choice(n, min(n, 64), replace=False)
    t1 = time.perf_counter()
    o1.site_pieces(pilot)
    dp = max(time.perf_counter() - t1, 1e-6)
    k = int(min(n, max(len(pilot), len(pilot) * one_thread_s / dp)))
    pick = rng.choice(n, k, replace=False)
    t1 = time.perf_counter()
    o1.site_pieces(pick)
    d1 = time.perf_counter() - t1
    o1.close()
    base = {"value": n / dt, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"whole workload: all {n} sites, every piece ({dt:.1f} s on {cores} threads)",
            "one_thread": {"value": k / d1, "unit": UNIT, "cores": 1,
                           "sample": f"all pieces of {k} random sites ({d1:.1f} s, 1 thread)"}}
    return base, op


def oracle_errors(w, res, op):
    """Measured errors of a computed result against the oracle's whole-workload
    pieces: per-site measure (relative), centroid (|dc| / |c| and |dc| / h_i with
    h_i = measure^(1/d)), and whether every site's neighbour list is identical."""
    import numpy as np

    n = len(w["sites"])
    keep = op.meas > 0
    oi = np.asarray(op.i, dtype=np.int64)
    om = np.zeros(n)
    m1 = np.zeros((n, 3))
    np.add.at(om, oi[keep], op.meas[keep])
    np.add.at(m1, oi[keep], op.m1[keep])
    oc = np.asarray(w["sites"], dtype=np.float64).copy()
    ok = om > 0
    oc[ok] += m1[ok] / om[ok, None]
    gm = res["measure"].double().cpu().numpy()
    gc = res["centroid"].double().cpu().numpy()
    rel = np.abs(gm[ok] - om[ok]) / om[ok]
    dc = np.linalg.norm(gc - oc, axis=1)
    dim = 3 if w["mode"] == 4 else 2
    h = om[ok] ** (1.0 / dim)
    # neighbours: unique bisector flags of faces of positive measure, per site
    cnt = np.diff(op.foff)
    own = np.repeat(np.arange(len(op.meas)), cnt)
    fl = np.asarray(op.flags, dtype=np.int64)
    sel = keep[own] & (fl >= 0)
    packed = np.unique((oi[own[sel]] << 32) | fl[sel])   # sorted unique (site, neighbour)
    pairs = np.stack([packed >> 32, packed & 0xFFFFFFFF], 1) if len(packed) else np.zeros((0, 2), np.int64)
    off = np.concatenate([[0], np.cumsum(np.bincount(pairs[:, 0], minlength=n))])
    same_nbr = bool(np.array_equal(res["nbr_off"].cpu().numpy(), off) and
                    np.array_equal(res["nbr_idx"].cpu().numpy().astype(np.int64), pairs[:, 1]))
    return {"sites_checked": int(n), "max_meas_rel": float(rel.max(initial=0)),
            "max_cent_rel": float((dc / np.maximum(np.linalg.norm(oc, axis=1), 1e-30)).max(initial=0)),
            "max_dc_over_h": float((dc[ok] / h).max(initial=0)), "empty_cells_match": bool(((gm > 0) == ok).all()),
            "neighbours_identical": same_nbr, "oracle_pieces": int(keep.sum()),
            "oracle_uncertain": int(op.stats.get("uncertain", 0))}


def serial_baseline(w, total_pieces, budget_s=8.0, seed=0):
    """The paper's serial method (Alg. 1 + Alg. 2) on one thread over a random
    sample of the simplices, scaled to the workload by its share of the pieces."""
    import numpy as np

    from paper_2509_07175_b300 import serial as S

    m = len(w["simp"])
    per_simplex = total_pieces / max(1, m)
    if per_simplex * 2e-4 > budget_s:   # one simplex alone is beyond the budget (~0.2 ms per piece)
        return {"value": None, "reason": f"{per_simplex:.0f} pieces per simplex: no bounded sample of whole simplices"}
    t0 = time.perf_counter()
    sv = S.Serial(w["mode"], w["sites"], w["verts"], w["simp"])
    setup = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    order = rng.permutation(m)
    done, pieces, t_run, k = 0, 0, 0.0, 1
    while done < m and t_run < budget_s:
        take = order[done:done + k]
        t1 = time.perf_counter()
        r = sv.run_list(take)
        t_run += time.perf_counter() - t1
        pieces += int((r.meas > 0).sum())
        done += len(take)
        per = t_run / done   # seconds per simplex so far: the next batch fits the rest of the budget
        k = int(max(1, min(2 * k, (budget_s - t_run) / max(per, 1e-9), m - done)))
    sv.close()
    frac = pieces / max(1, total_pieces)
    est = setup + t_run / max(frac, 1e-12)
    return {"value": len(w["sites"]) / est, "unit": UNIT, "cores": 1, "kind": "serial Alg. 1 + Alg. 2 (C, FP64)",
            "sample": f"{done} random simplices of {m} ({pieces} of {total_pieces} pieces, {t_run:.1f} s), "
                      f"setup {setup:.2f} s; cells/s = sites / (setup + sample time / piece share)"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on the host cores.  Each step
    computes every piece of a random sample of the workload's sites, sized so that
    the whole run stays within a few minutes; ms_per_step is that step's time."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from paper_2509_07175_b300 import inputs as I

    w = I.workload(args.workload)
    n = len(w["sites"])
    cores = os.cpu_count() or 1
    o = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"], nthreads=cores)
    rng = np.random.default_rng(0)
    step_s = min(10.0, max(1.0, 90.0 / max(1, args.steps + args.warmup)))
    pilot = rng.choice(n, min(n, 16 * cores), replace=False)
    t0 = time.perf_counter()
    o.site_pieces(pilot)
    dp = max(time.perf_counter() - t0, 1e-6)
    k = int(min(n, max(len(pilot), len(pilot) * step_s / dp)))
    times = []
    for step in range(args.warmup + args.steps):
        pick = rng.choice(n, k, replace=False)
        t0 = time.perf_counter()
        o.site_pieces(pick)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    o.close()
    ms = 1e3 * statistics.median(times)
    value = k / (ms / 1e3)
    base = {"value": value, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"each step: all pieces of {k} random sites of the {n} ({ms / 1e3:.2f} s)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": DESC.get(args.workload), "n_sites": n,
                       "n_simplices": len(w["simp"]), "sites_per_step": k},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(DESC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain", action="store_true", help="time the plain search instead of the learned form")
    ap.add_argument("--topk", type=int, default=24)
    ap.add_argument("--proposal", default="mlp", choices=["mlp", "distance"],
                    help="ranking of the 32 nearest sites in the learned form")
    ap.add_argument("--split", default="on", choices=["on", "off"],
                    help="3D tetrahedra: interior sites' cells whole after the boundary pass (Alg. 5)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch

    from paper_2509_07175_b300 import binding as B
    from paper_2509_07175_b300 import inputs as I

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    training = None
    mlp = not args.plain and args.proposal == "mlp"
    if mlp:
        # the learned proposal's network, trained on the GPU on labels the method
        # produces for seeded 100k-site cube instances (outside the timed region)
        from paper_2509_07175_b300 import learned as L
        training = L.trained_state(mix=L.MIX)
    w = I.workload(args.workload)
    n = len(w["sites"])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    d = B.diagram_from_workload(w)
    # device memory of one context: its inputs, the library's buffers and one
    # computation's pair set and outputs (cudaMemGetInfo before and after)
    code, _r = d.compute_raw()
    assert code == 0, B.ERRORS.get(code, code)
    torch.cuda.synchronize()
    device_memory = {"bytes": int(free0 - torch.cuda.mem_get_info()[0]),
                     "note": "cudaMemGetInfo difference from before the context to after its first compute"}
    device_memory["bytes_per_site"] = device_memory["bytes"] / n
    if mlp:
        L.load_state(d, training["state"])
    prop = B.PROPOSAL_MLP if mlp else B.PROPOSAL_DISTANCE
    split = int(args.split == "on" and w["mode"] == B.MODE_3D and w.get("box") is None)
    form = dict(learned=0 if args.plain else 1, topk=args.topk, proposal=prop, split=split)
    relax = None
    if w.get("lloyd"):
        # blue noise (Sec. 6.4): relax the sites by graph-captured Lloyd iterations
        # of the timed form first; the iterations are timed as a whole
        d.set_options(mapping=0, **form)
        d.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.lloyd(int(w["lloyd"]), use_graph=True)
        torch.cuda.synchronize()
        relax = {"iters": int(w["lloyd"]), "s": time.perf_counter() - t0,
                 "note": "graph-captured Lloyd iterations (compute + centroid update) from the white-noise sites, "
                         "list size and mapping tuned on the white-noise sites"}
        w = dict(w, sites=d.sites().double().cpu().numpy())
        d.close()
        d = B.diagram_from_workload(w)
        if mlp:
            L.load_state(d, training["state"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    owner_t = ex = None
    if world > 1:
        # one diagram across the ranks: each computes the cells of its own sites
        from paper_2509_07175_b300 import parallel as P
        owner_t = torch.tensor(P.morton_owner(w["sites"], world), device="cuda")
        d.set_partition(owner_t, rank)
        ex = P.DistExchange(dist, rank, world, "cuda")

    def step():
        """One step: (status, clip-phase ms, kernels launched)."""
        if ex is None:
            code, r = d.compute_raw()
            return code, r.phase_ms[3], int(r.stats[13])
        res, _rounds = P.compute(d, owner_t, ex)
        return res["status"], res["phase_ms"]["clip"], int(res["stats"].get("launches", 0))

    def time_form(opts, steps, warm=2):
        """Median ms per step of a form (L2 flushed before each step, CUDA events)."""
        d.set_options(**opts)
        for _ in range(warm):
            code = step()[0]
            assert code == 0, B.ERRORS.get(code, code)
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            code = step()[0]
            e1.record(stream)
            torch.cuda.synchronize()
            assert code == 0, B.ERRORS.get(code, code)
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    # the plain form (the paper's search alone) and the learned form with the
    # distance ranking beside the headline form: identical output, timed the same way
    beside = {}
    network = None
    if not args.plain:
        d.set_options(learned=0, split=split)
        ref = d.compute()
        if mlp:
            # what the network ranks on this workload: recall of the neighbours among
            # its top k of the 32 nearest, against the ranking by distance
            x, yv = d.mlp_features()
            z = d.mlp_forward(x)
            zd = -torch.arange(32, device="cuda", dtype=torch.float32).expand(x.shape[0], 32)
            network = {"recall_at_k": {str(k): {"network": L.recall_at_k(z, yv, k),
                                                "distance": L.recall_at_k(zd, yv, k)} for k in (4, 8, 16, 24)},
                       "rows": int(x.shape[0])}
            del x, yv, z, zd
        nb = max(1, min(5, args.steps))
        beside["plain"] = time_form(dict(learned=0, split=split), nb)
        if mlp:
            beside["learned_distance"] = time_form(dict(learned=1, topk=args.topk, split=split,
                                                        proposal=B.PROPOSAL_DISTANCE), nb)
    # counters for the roofline numerator (an untimed run with the counters on)
    d.set_options(stats=1, **form)
    rs = d.compute()
    counts = rs["stats"]
    if not args.plain:
        for key in ("measure", "centroid", "nbr_off", "nbr_idx"):
            assert torch.equal(ref[key], rs[key]), f"learned form differs from plain in {key}"
    # batching: the autotuner times every clip-kernel mapping (warp / thread per pair x
    # queue chunk) on this workload and caches the fastest for the timed steps
    d.set_options(timing=1, mapping=0, **form)
    tune = d.autotune()
    for _ in range(args.warmup):
        code = step()[0]
        assert code == 0, B.ERRORS.get(code, code)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clip_ms = []
    launches = 0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        code, cms, nl = step()
        ends[k].record(stream)
        assert code == 0, B.ERRORS.get(code, code)
        clip_ms.append(cms)
        launches += nl
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    (total_ms,), (launches,) = reduce_over_ranks(dist, [sum(step_ms)], [launches], "cuda")
    launches = int(launches)
    # one diagram of n cells per step, over the slowest rank's time
    value = whole_job_rate(n, args.steps, total_ms)

    # end to end through the public API with host buffers
    dim = 2 if w["mode"] == B.MODE_2D else 3
    dt = torch.float64 if w["f64"] else torch.float32
    host_sites = torch.tensor(w["sites"][:, :dim], dtype=dt).pin_memory()
    meas_h = torch.empty(n, dtype=dt).pin_memory()
    cen_h = torch.empty((n, 3), dtype=dt).pin_memory()
    off_h = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    nnz = int(rs["nbr_off"][-1].item())
    idx_h = torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory()
    d.set_options(**form)
    for _ in range(2):
        d.update_sites_host(host_sites)
        step()
        d.copy_result_host(meas_h, cen_h, off_h, idx_h)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d.update_sites_host(host_sites)
        step()
        d.copy_result_host(meas_h, cen_h, off_h, idx_h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    (e2e_s,), _ = reduce_over_ranks(dist, [e2e_s], [], "cuda")
    e2e_val = whole_job_rate(n, args.steps, e2e_s * 1e3)
    esz = 8 if w["f64"] else 4
    h2d = n * dim * esz
    d2h = n * esz + 3 * n * esz + (n + 1) * 8 + nnz * 4

    if rank != 0:
        d.close()
        if dist:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    sm = 148
    try:
        sm = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        pass
    max_mhz = ck.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0)
    peak_tflops = sm * 128 * 2 * max_mhz * 1e6 / 1e12
    # 8 FLOP per site-distance evaluation: grid scans plus the 32-site list tests
    flops = 8.0 * (counts["sites_scanned"] + 32 * counts.get("list_tests", 0))
    clip_s = statistics.median(clip_ms) / 1e3 if clip_ms else float("nan")
    achieved = flops / clip_s / 1e12
    nnz_all = int(rs["nbr_off"][-1].item())
    hbm_bytes = 16.0 * n + 4.0 * n + 12.0 * n + 8.0 * (n + 1) + 4.0 * nnz_all
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64" if w["f64"] else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": DESC[args.workload], "n_sites": n,
                   "n_simplices": len(w["simp"]), "pairs": counts["pairs"], "nonempty_pieces": counts["nonempty"],
                   "split": ({"whole_cells": counts["whole_cells"], "boundary_sites": counts["boundary_sites"]}
                             if split else None),
                   "l2": "flushed before every step (256 MiB write, outside the timed events)",
                   "parallelism": f"site partition x{world} (Morton ranges)" if world > 1 else "single GPU"},
        "roofline": {"kernel": "k_flood<float, 3D> (Alg. 3 clip + flood)", "bound": "alu", "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "peak_source": f"{sm} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz (derived)",
                     "limiter": "latency (dependent shared-memory, warp-vote and L2 chains at 12 warps per SM); "
                                "neither roof is approached",
                     "hbm": {"achieved": (hbm_bytes / clip_s / 1e9) if hbm_bytes else None,
                             "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                             "frac": (hbm_bytes / clip_s / 1e9 / peaks["hbm_gbs"])
                             if hbm_bytes and peaks.get("hbm_gbs") else None,
                             "bytes": hbm_bytes, "note": "algorithmic bytes per launch: 100 B per cell x sites "
                                                         "(site read 16, measure 4, centroid 12, CSR offset 8, "
                                                         "neighbour ids 4 x degree)"},
                     "flops_per_launch": flops, "clip_ms": clip_s * 1e3,
                     "clip_share": (clip_s * 1e3) / (total_ms / args.steps),
                     "traffic": flood_traffic(args.workload),
                     "traffic_note": "dram bytes per launch of the 3D clip kernel, single-pass ncu capture of "
                                     "the same kernel (learned form, distance ranking, top 24, split as timed); "
                                     "null once the kernel sources differ from the captured ones"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "device_memory": device_memory,
        "autotune": {"choice": ("warp" if tune["mapping"] == 1 else "thread") + f" per pair, chunk {tune['chunk']}",
                     "clip_ms_by_candidate": tune["times_ms"]},
        "clocks": ck,
        "stats": {k: counts[k] for k in ("nn_queries", "corner_tests", "clips", "lambda_steps", "search_steps",
                                         "fp64", "uncertain", "ties", "sites_scanned", "fallback", "learned_hits",
                                         "list_tests", "bisector_faces", "excess_clips")},
        "form": ("plain (Sec. 3.2 / 5.1 search)" if args.plain else
                 f"learned+batched ({args.proposal} ranking of the 32 nearest, top-{args.topk}; "
                 "output bit-identical to plain)") + ("; Alg. 5 split (interior cells whole)" if split else ""),
    }
    step_med = statistics.median(step_ms)
    for name, ms in beside.items():
        line[name] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                      "speedup_headline_over_this": ms / step_med}
    if training is not None:
        line["training"] = {"rows": training["rows"], "epochs": training["epochs"], "batch": training["batch"],
                            "lr": training["lr"], "train_s": training["train_s"], "data_s": training["data_s"],
                            "loss_first_epoch": training["epoch_loss"][0],
                            "loss_last_epoch": training["epoch_loss"][-1],
                            "data": "labels from plain computes of seeded 100k-site instances: "
                                    + ", ".join(f"{c} {nm}" for nm, c in L.MIX)}
        if network is not None:
            line["network"] = network
    if relax is not None:
        line["lloyd_relaxation"] = relax
    if world == 1 and not args.no_cpu_baseline and relax is not None:
        line["cpu_baseline"] = {"value": None, "reason": "the relaxed sites come from this library's own Lloyd "
                                                         "iterations; the oracle is not fed from the CUDA path "
                                                         "(blue100k checks blue noise against it)"}
    elif world == 1 and not args.no_cpu_baseline:
        base, op = cpu_baseline(w)
        line["cpu_baseline"] = base
        line["oracle_check"] = oracle_errors(w, rs, op)
        line["serial_baseline"] = serial_baseline(w, total_pieces=int((op.meas > 0).sum()))
        del op
    d.close()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
