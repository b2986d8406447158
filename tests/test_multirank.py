"""The bench's multi-rank path on the CPU (gloo, 2 ranks): each rank runs its
own realisation, the job time is the slowest rank's, the value sums the
particles of all ranks; a rank's seed differs from the others'."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    total = bench.max_over_ranks(local_ms, device="cpu")
    value = bench.job_throughput(world, 1000, 10, total)
    seeds = [None] * world
    w = bench.make_workload("plummer", rank)
    dist.all_gather_object(seeds, float(w["pos"][0, 0]))
    out[rank] = (total, value, seeds)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        total, value, seeds = out[r]
        assert total == 150.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)
        assert seeds[0] != seeds[1]
