"""The multi-GPU path of bench.py is replicas only (independent seeded
instances, no data-path collective); its host logic -- per-rank instance seeds,
max-over-ranks timing and summed counts -- runs here as two gloo ranks on CPU."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    from paper_2509_07175_b300 import inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_ms = [100.0 + 10 * rank, 50.0]
    maxes, sums = bench.reduce_over_ranks(dist, [sum(step_ms), 1.5 * rank], [7 + rank, 1], "cpu")
    seed = bench.replica_seed(rank)
    w = I.workload("cube", 2000, seed=seed)
    q.put((rank, maxes, sums, seed, float(w["sites"][:, 0].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, s0, seed0, x0), (r1, m1, s1, seed1, x1) = out
    # every rank sees the slowest rank's time and the summed counts
    assert m0 == m1 == [160.0, 1.5]
    assert s0 == s1 == [15.0, 2.0]
    # independent instances: rank 0 the workload's own seed, rank 1 another one
    assert seed0 is None and seed1 is not None and x0 != x1


def test_single_process_reduction_and_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, [3.0], [4], "cpu") == ([3.0], [4])
    # 1,000,000 cells x 10 steps x 2 ranks in 5 s of the slowest rank
    assert bench.whole_job_rate(1_000_000, 10, 2, 5000.0) == pytest.approx(4e6)
