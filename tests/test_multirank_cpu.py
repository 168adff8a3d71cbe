"""The multi-rank (N > 1) host logic of bench.py on CPU with the gloo backend.

Each rank advances its own replica (no data-path collective); the timed
region's duration is the maximum over ranks and the whole-job rate counts
every rank's cells."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
    ms_max = bench.reduce_max(local_ms, dist, "cpu")
    rate = bench.aggregate_rate(1000, 4, world, ms_max * 1e-3)
    q.put((rank, ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 15.0
        assert abs(rate - world * 1000 * 4 / 0.015 / 1e9) < 1e-15
