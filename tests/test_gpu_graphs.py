"""The stream-ordered entry points can be captured into a CUDA graph and
replayed: rank, rank_4 and the persistent QuadFm count (whose work-queue
counter comes from the stream-ordered pool, i.e. memory nodes in the graph)."""
import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth
from tests.gpu_util import dev_u64, dev_u8, host_u64

pytestmark = pytest.mark.gpu


def test_rank_in_cuda_graph():
    import torch
    from paper_2602_04103_gb300 import capi
    torch.cuda.set_device(0)
    for layout in (0, 1):
        n = 3 * 63488 + 17
        words = synth.bits(301, n, 0.5)
        idx = capi.qr_build(dev_u64(words), n, 2, layout=layout)
        q = synth.queries(302, n, 100_000)
        dq = dev_u64(q)
        out = torch.empty_like(dq)
        capi.qr_rank(idx, dq, 1, out)          # first call outside capture (caches launch shapes)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            capi.qr_rank(idx, dq, 1, out)
        for _ in range(2):
            out.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(host_u64(out), oracle.rank(words, n, 2, q, 1)[0])
        n4 = 2 * 57344 + 5
        w4 = synth.dna_uniform(303, n4)
        idx4 = capi.qr_build(dev_u64(w4), n4, 4, layout=layout)
        q4 = synth.queries(304, n4, 50_000)
        dq4 = dev_u64(q4)
        o4 = torch.empty((q4.size, 4), dtype=torch.int64, device="cuda")
        capi.qr_rank4(idx4, dq4, o4)
        torch.cuda.synchronize()
        g4 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g4):
            capi.qr_rank4(idx4, dq4, o4)
        o4.fill_(-1)
        g4.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host_u64(o4).reshape(-1, 4), oracle.rank4(w4, n4, q4)[0])


def test_qfm_count_in_cuda_graph():
    import torch
    from paper_2602_04103_gb300 import capi
    torch.cuda.set_device(0)
    n = 1 << 18
    t = synth.fm_text(311, n, repeat_cover=0.2, len_min=300, len_max=2000, sub_rate=0.02)
    idx = capi.qfm_build(dev_u8(t), n)
    pats, off = synth.patterns(312, t, 20_000, 1, 120, 0.01)
    dp, doff = dev_u8(pats), dev_u64(off)
    out = torch.empty(off.size - 1, dtype=torch.int64, device="cuda")
    capi.qfm_count(idx, dp, doff, out)
    torch.cuda.synchronize()
    want = host_u64(out).copy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        capi.qfm_count(idx, dp, doff, out)
    for _ in range(3):                          # the queue counter is reset inside the graph
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host_u64(out), want)
    sample = np.arange(0, off.size - 1, 97)
    sub = np.concatenate([pats[off[k]:off[k + 1]] for k in sample])
    sub_off = np.concatenate([[0], np.cumsum((off[sample + 1] - off[sample]).astype(np.int64))]).astype(np.uint64)
    assert np.array_equal(want[sample], oracle.count_brute_batch(t, sub, sub_off))


@pytest.mark.parametrize("mode", ["regions", "auto"])
def test_region_batching_in_cuda_graph(mode):
    """Region batching under capture: its scratch becomes a graph memory node,
    and the probe of the automatic rule runs inside the graph."""
    import torch
    from paper_2602_04103_gb300 import capi
    torch.cuda.set_device(0)
    if mode == "regions":
        n, m = 3 * 63488 + 17, 3 * 8192 + 5
    else:
        n, m = 1 << 30, 1 << 22          # 143 MB index, 2^22 queries: the automatic rule picks region batching
    words = synth.bits(321, n, 0.5)
    q = synth.queries(322, n, m)
    idx = capi.qr_build(dev_u64(words), n, 2, layout=1)
    if mode == "regions":
        capi.qr_set_batch_mode(idx, capi.QR_BATCH_REGIONS)
    assert capi.qr_rank_plan(idx, m) == capi.QR_BATCH_REGIONS
    dq = dev_u64(q)
    out = torch.empty_like(dq)
    capi.qr_rank(idx, dq, 1, out)          # first call outside capture (per-device set-up)
    torch.cuda.synchronize()
    want = host_u64(out).copy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        capi.qr_rank(idx, dq, 1, out)
    for _ in range(2):
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host_u64(out), want)
    sample = np.arange(0, m, 101)
    assert np.array_equal(want[sample], oracle.rank(words, n, 2, q[sample], 1)[0])
    assert capi.qr_status(idx) == 0
