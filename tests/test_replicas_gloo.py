"""The bench's multi-GPU mode runs independent replicas (the path has no data
exchange to shard): each rank times its own copy, the job time is the slowest
rank's, and the rate counts every rank's work.  Checked here with two gloo ranks
on the CPU."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        total = bench.max_over_ranks(10.0 * (rank + 1), dist)   # rank 1 is the slow one
        rate = bench.whole_job_rate(1000, ws, 4, total)
        out.put((rank, ws, r, local, total, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r0, ws, r, local, total, rate) in enumerate(res):
        assert (r0, ws, r, local) == (rank, 2, rank, rank)
        assert total == 20.0
        assert rate == pytest.approx(2 * 1000 * 5 * 4 / 0.020)


def test_single_process_defaults():
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench._dist() == (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                             int(os.environ.get("LOCAL_RANK", "0")))
