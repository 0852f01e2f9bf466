"""The multi-rank path of bench.py on CPU (gloo, world size 2).

Every rank advances its own seeded replica of the workload and the job's
time is the slowest rank's; these tests check the rank plumbing (seeds,
max over ranks, barrier, whole-job throughput) without a GPU.
"""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank                    # rank 1 is the slower one
        bench.barrier(world)
        worst = bench.max_over_ranks(ms, world)
        args = type("A", (), {"nx": 512, "ny": 256, "nz": 256, "steps": 10})()
        sc = bench.workload(args, rank)
        q.put((rank, worst, [b.pos for b in sc.bodies][:1],
               bench.job_mlups(sc.cells, 10, world, worst)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_use_distinct_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == out[1][1] == 150.0
    assert out[0][2] != out[1][2]                   # seeds differ per rank
    cells = 512 * 256 * 256
    assert out[0][3] == pytest.approx(cells * 10 * 2 / 0.15 / 1e6)
