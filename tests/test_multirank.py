"""The N > 1 path of bench.py: independent replicas, a barrier, the max over ranks of
the timed region and whole-job throughput, exercised with world_size 2 on gloo (CPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    mx = bench.reduce_max(ms)
    rate = bench.whole_job_rate(5, world, mx)
    out.put((rank, mx, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == 150.0
    assert abs(res[0][2] - 2 * 5 / 0.150) < 1e-9


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_rate(4, 1, 200.0) == 20.0
