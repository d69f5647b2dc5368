"""The multi-GPU form is replicas only (independent streams per rank, no
exchange step).  Its one cross-rank step, the job throughput from per-rank
times and units, runs here on CPU with two gloo ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 * (r + 1) ms for 5 + r frames
        value, max_ms, total = bench.combine_ranks(10.0 * (rank + 1), 5 + rank, dist=dist)
        dist.barrier()
        q.put((rank, value, max_ms, total))
    finally:
        dist.destroy_process_group()


def test_two_replicas_combine_by_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, max_ms, total in res:
        assert max_ms == 20.0 and total == 11.0
        assert value == pytest.approx(11.0 / 0.020)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    value, max_ms, total = bench.combine_ranks(8.0, 16)
    assert (max_ms, total) == (8.0, 16.0) and value == pytest.approx(2000.0)
