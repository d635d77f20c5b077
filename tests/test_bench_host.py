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


def test_region_pass_bytes():
    """Algorithmic bytes per query of the region passes: 8 (q) + 4 (key) + 2
    (index) + two segment tables in the sort; 4 + 4 + one table + the index
    once per batch in the rank pass; 4 + 2 + one table + 8 in the unsort
    (rank_4: 16-byte results and 32-byte rows)."""
    import bench
    seg = 4 * 256 / 8192
    m, idx = 1 << 28, 2_291_767_764
    b = bench.region_pass_bytes(m, idx)
    assert b == {"sort": 14 + 2 * seg, "rank": 8 + seg + idx / m, "unsort": 14 + seg}
    assert abs(sum(b.values()) - 45.0375) < 1e-3                  # the BiRank headline step
    b4 = bench.region_pass_bytes(m, idx, rank4=True)
    assert b4["rank"] == 20 + seg + idx / m and b4["unsort"] == 50 + seg
    assert bench.region_pass_bytes(m, idx, per_query_c=True)["sort"] == 15 + 2 * seg
    # the QuadFm step: two rank queries of a QuadRank16 line, lower half one sector,
    # upper half the 16 delta bytes and one sector
    assert abs(2 * bench.QFM_RANK_L2_BYTES - 82.2857) < 1e-3


def test_parse_cpulist():
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("72-143") == set(range(72, 144))
    assert bench.parse_cpulist("") == set()
