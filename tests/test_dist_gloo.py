"""Multi-process (world size 2, gloo, CPU) checks of the benchmark's N > 1
logic: ranks solve independent problem instances (distinct seeds, no data
exchange) and the job time is the maximum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        c = bench.cfg()
        seed = bench.replica_seed(c["seed"], rank)
        elapsed = 1.0 + rank          # rank 1 is the slow one
        m = bench.max_over_ranks(elapsed, world)
        v = bench.job_throughput(600 * 4, world, m)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        q.put((rank, m, v, seeds))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, seeds in out:
        assert m == 2.0                                  # slowest rank's time
        assert v == pytest.approx(2 * 600 * 4 / 2.0)     # all ranks' units / that time
        assert len(set(seeds)) == 2                      # independent problems
