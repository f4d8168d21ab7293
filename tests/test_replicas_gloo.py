"""The N > 1 path of the bench on CPU: two gloo ranks (world_size 2) take the
replica seeds and the max-over-ranks timing reduction that the GPU run uses
over NCCL.  Replicas solve independent seeded instances, so the timing
all-reduce is the only collective."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_20174_gb300 import inputs as gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.replica_seed(bench.WL["seed"], rank)
        p = gen.poisson_2d(8, 2, 4, seed=seed)
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        total = bench.max_over_ranks(local_ms, world, "cpu")
        rate = bench.whole_job_rate(world, 4, total)
        out[rank] = (seed, float(p.f[0, 0]), total, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_timing_and_distinct_instances():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, f0, t0, r0), (s1, f1, t1, r1) = res[0], res[1]
    assert s0 != s1 and f0 != f1          # independent seeded instances
    assert t0 == t1 == 150.0              # both ranks see the slowest rank's time
    assert r0 == r1 == pytest.approx(2 * 4 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(1, 5, 1000.0) == pytest.approx(5.0)
