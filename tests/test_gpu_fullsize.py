"""Full-size parity at the benchmark's sizes and launch configuration (the
tuned build of workloads.build_tuned): the GPU answers every query, and a
sample of outputs is checked against the oracle bit-exactly.

* BiRank: n = 2^34 bits (p = 0.5 and 0.01), 2^28 uniform queries, and the
  same queries sorted; 2^20 sampled outputs per case, both symbols.
* QuadRank: n = 2^32 chars (uniform, GC + runs), 2^28 queries, rank with
  random symbols and rank_4 on 2^20 sampled queries.
* QuadFm: 2^26-char text, 10^7 patterns: persistent counts equal the
  per-step baseline on every pattern and brute-force counts on a sample.
"""
import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import workloads
from tests.gpu_util import dev_u64, dev_u8, host_u64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.empty_cache()


@pytest.mark.parametrize("p,sorted_q", [(0.5, False), (0.01, False), (0.5, True)])
def test_birank_full_size(p, sorted_q):
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 34
    text, q = workloads.birank_inputs(34, 28, p=p)
    dq = dev_u64(q)
    if sorted_q:
        dq = torch.sort(dq).values       # uniform queries, sorted ascending
        q = host_u64(dq)
    idx, layout, _ = workloads.build_tuned(dev_u64(text), n, 2, dq, c=1)
    out = torch.empty_like(dq)
    sample = workloads.sample_indices(q.size, 1 << 20, 5)
    for c in (1, 0):
        capi.qr_rank(idx, dq, c, out)
        got = host_u64(out)[sample]
        want, rc = oracle.rank(text, n, 2, q[sample], c)
        assert rc == 0 and np.array_equal(got, want), (layout, c)
    # the other batch path (region batching or the direct kernels) agrees on every output
    plan = capi.qr_rank_plan(idx, q.size)
    capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT if plan == capi.QR_BATCH_REGIONS else capi.QR_BATCH_REGIONS)
    other = torch.empty_like(dq)
    capi.qr_rank(idx, dq, 0, other)
    assert torch.equal(other, out), (layout, plan)
    assert capi.qr_status(idx) == 0
    idx.free()


@pytest.mark.parametrize("kind", ["uniform", "gc_runs"])
def test_quadrank_full_size(kind):
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 32
    text, q, c = workloads.quadrank_inputs(32, 28, kind)
    dq, dc = dev_u64(q), dev_u8(c)
    idx, layout, _ = workloads.build_tuned(dev_u64(text), n, 4, dq, c=dc)
    out = torch.empty_like(dq)
    capi.qr_rank_c(idx, dq, dc, out)
    sample = workloads.sample_indices(q.size, 1 << 20, 6)
    want, rc = oracle.rank_c(text, n, 4, q[sample], c[sample])
    assert rc == 0 and np.array_equal(host_u64(out)[sample], want)
    plan = capi.qr_rank_plan(idx, q.size)
    capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT if plan == capi.QR_BATCH_REGIONS else capi.QR_BATCH_REGIONS)
    other = torch.empty_like(dq)
    capi.qr_rank_c(idx, dq, dc, other)
    assert torch.equal(other, out), (layout, plan)
    capi.qr_set_batch_mode(idx, capi.QR_BATCH_AUTO)
    del out, other
    out4 = torch.empty((q.size, 4), dtype=torch.int64, device="cuda")
    capi.qr_rank4(idx, dq, out4)
    want4, _ = oracle.rank4(text, n, q[sample])
    assert np.array_equal(host_u64(out4).reshape(-1, 4)[sample], want4)
    assert capi.qr_status(idx) == 0
    idx.free()


def test_fm_full_size():
    import torch
    from paper_2602_04103_gb300 import capi
    text, pats, off = workloads.fm_inputs()
    m = off.size - 1
    idx = capi.qfm_build(dev_u8(text), text.size)
    dp, doff = dev_u8(pats), dev_u64(off)
    a = torch.empty(m, dtype=torch.int64, device="cuda")
    b = torch.empty(m, dtype=torch.int64, device="cuda")
    capi.qfm_count(idx, dp, doff, a)
    capi.qfm_count_stepwise(idx, dp, doff, b)
    got = host_u64(a)
    assert np.array_equal(got, host_u64(b))
    sample = workloads.sample_indices(m, 256, 7)
    sub = np.concatenate([pats[off[k]:off[k + 1]] for k in sample])
    sub_off = np.concatenate([[0], np.cumsum((off[sample + 1] - off[sample]).astype(np.int64))]).astype(np.uint64)
    assert np.array_equal(got[sample], oracle.count_brute_batch(text, sub, sub_off))
    # invariants over every pattern: a count never exceeds the number of start positions
    lens = (off[1:] - off[:-1]).astype(np.int64)
    assert (got.astype(np.int64) <= text.size - lens + 1).all()
    assert capi.qfm_status(idx) == 0
    idx.free()
