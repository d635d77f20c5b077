"""Host-side logic of bench.py: the max-over-ranks reduction of the timed
region on two gloo ranks (CPU), and the per-query accounting."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(10.0 + rank, world, device="cpu")
    q.put((rank, got))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 11.0, 1: 11.0}


def test_bytes_and_requests_per_query():
    import bench
    assert bench.bytes_per_query(2, 0, 0) == 80          # 64-byte line + q + out
    assert bench.bytes_per_query(2, 1, 0) == 48          # 32-byte sector + q + out
    assert bench.bytes_per_query(4, 1, 0, rank4=True) == 72
    assert bench.requests_per_query(2, 1, 0) == 1.0 and bench.requests_per_query(2, 2, 0) == 1.0
    assert bench.bytes_per_query(2, 2, 0) == 144
    assert bench.requests_per_query(2, 0, 2) == 2.0
    assert bench.requests_per_query(2, 0, 4) == 1.0 and bench.requests_per_query(4, 0, 4) == 1.0
    assert abs(bench.requests_per_query(2, 0, 3) - (240 / 496 + 2 * 256 / 496)) < 1e-12
