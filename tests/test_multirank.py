"""The benchmark's multi-rank bookkeeping on CPU with two gloo ranks (replicas: every rank
solves its own problems; the job's time is the slowest rank's)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" (r + 1) * 10 ms for 1e6 unknowns
    slowest = bench.max_over_ranks((rank + 1) * 0.010, dist)
    value = bench.job_throughput(1_000_000, world, slowest)
    t = torch.tensor([slowest, value], dtype=torch.float64)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t)
    if rank == 0:
        out.put([g.tolist() for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for slowest, value in res:
        assert slowest == pytest.approx(0.020)
        assert value == pytest.approx(2 * 1_000_000 / 0.020)


def test_single_process_path_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, None) == 0.5
    assert bench.job_throughput(10, 1, 2.0) == 5.0
