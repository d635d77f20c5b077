"""Full-size parity at the benchmark's sizes and launch configuration (the
tuned build of workloads.build_tuned): the GPU answers every query, and a
sample of outputs is checked against the oracle bit-exactly.

* BiRank: n = 2^34 bits (p = 0.5 and 0.01), 2^28 uniform queries, and the
  same queries sorted; 2^20 sampled outputs per case, both symbols.
* QuadRank: n = 2^32 chars (uniform, GC + runs), 2^28 queries, rank with
  random symbols and rank_4 on 2^20 sampled queries; region batching and
  the direct kernels agree on every output of both.
* QuadFm count (2^26-char text, 10^7 patterns): the GPU suffix array row by
  row, all 10^7 counts and the reverse-complement counts of 10^5 sampled
  patterns against the oracle (tests/golden/fm_full_2p26_1e7.json holds
  sha256 digests of the oracle's arrays, written by make_fm_full.py, which
  calls only the oracle; on a mismatch the oracle is run here to name the
  first differing row), plus the per-step baseline on every pattern.
* QuadFm serving (2^28-char text): 256 requests (489,363 patterns) served by
  the continuous-batching server; 2000 sampled counts against the oracle's
  brute-force counts (tests/golden/fm_serving_2p28.json).
"""
import hashlib
import json
from pathlib import Path

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
    # rank_4 by the other batch path agrees on every output
    plan4 = capi.qr_rank_plan(idx, q.size, 1)
    capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT if plan4 == capi.QR_BATCH_REGIONS else capi.QR_BATCH_REGIONS)
    other4 = torch.empty_like(out4)
    capi.qr_rank4(idx, dq, other4)
    assert torch.equal(other4, out4), (layout, plan4)
    assert capi.qr_status(idx) == 0
    idx.free()


GOLDEN = Path(__file__).resolve().parent / "golden"


def sha(a: np.ndarray, dtype: str) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def first_diff(got: np.ndarray, want: np.ndarray):
    bad = np.flatnonzero(got != want)
    return (int(bad.size), bad[:5].tolist(), got[bad[:5]].tolist(), want[bad[:5]].tolist())


def test_fm_full_size():
    import torch
    from paper_2602_04103_gb300 import capi
    g = json.loads((GOLDEN / "fm_full_2p26_1e7.json").read_text())
    text, pats, off = workloads.fm_inputs()
    m = off.size - 1
    assert (text.size, m) == (g["n"], g["patterns"])
    idx = capi.qfm_build(dev_u8(text), text.size, capi.QFM_KEEP_SA)
    # the suffix array of T$, row by row
    sa = torch.empty(text.size + 1, dtype=torch.int32, device="cuda")
    capi.qfm_export(idx, sa=sa)
    sa_h = sa.cpu().numpy().view(np.uint32)
    if sha(sa_h, "<u4") != g["sa_uint32_sha256"]:
        want = oracle.suffix_array(text).astype(np.uint32)
        assert False, ("suffix array differs from the oracle's", first_diff(sa_h, want))
    del sa
    # all 10^7 counts
    dp, doff = dev_u8(pats), dev_u64(off)
    a = torch.empty(m, dtype=torch.int64, device="cuda")
    capi.qfm_count(idx, dp, doff, a)
    got = host_u64(a)
    if sha(got, "<u8") != g["counts_uint64_sha256"]:
        want = oracle.count_sa(text, oracle.suffix_array(text), pats, off)
        assert False, ("counts differ from the oracle's", first_diff(got, want))
    assert int(got.sum()) == g["counts_sum"] and int((got == 0).sum()) == g["counts_zero"]
    # the per-step baseline gives the same counts
    b = torch.empty(m, dtype=torch.int64, device="cuda")
    capi.qfm_count_stepwise(idx, dp, doff, b)
    assert torch.equal(a, b)
    del b
    # both strands: the forward half again, the reverse complements on the sample
    ab = torch.empty(2 * m, dtype=torch.int64, device="cuda")
    capi.qfm_count_ex(idx, dp, doff, ab, capi.QFM_BOTH_STRANDS)
    assert torch.equal(ab[:m], a)
    ids = workloads.sample_indices(m, 100_000, 41)
    assert ids.size == g["revcomp_sample"]["size"]
    rc_got = host_u64(ab[m:])[ids]
    if sha(rc_got, "<u8") != g["revcomp_sample"]["counts_uint64_sha256"]:
        sub = np.concatenate([pats[int(off[k]):int(off[k + 1])] for k in ids])
        sub_off = np.concatenate([[0], np.cumsum((off[ids + 1] - off[ids]).astype(np.int64))]).astype(np.uint64)
        want = oracle.count_sa(text, oracle.suffix_array(text), oracle.revcomp_batch(sub, sub_off), sub_off)
        assert False, ("reverse-complement counts differ", first_diff(rc_got, want))
    # invariants over every pattern: a count never exceeds the number of start positions
    lens = (off[1:] - off[:-1]).astype(np.int64)
    assert (got.astype(np.int64) <= text.size - lens + 1).all()
    assert capi.qfm_status(idx) == 0
    idx.free()


def test_fm_serving_full_size():
    """The serving workload at its size: a 2^28-char index resident on the
    device, 256 requests of 1..4096 patterns served by the continuous-batching
    server (4 slots, every request submitted at once, so they share batches);
    2000 sampled counts equal the oracle's brute-force counts, and every count
    equals a plain qfm_count over the whole trace."""
    import torch
    from paper_2602_04103_gb300 import capi
    g = json.loads((GOLDEN / "fm_serving_2p28.json").read_text())
    text, pats, off, first = workloads.serving_inputs(g["requests"], 28)
    npat = int(first[-1])
    assert (text.size, npat) == (g["n"], g["patterns"])
    idx = capi.qfm_build(dev_u8(text), text.size)
    del text
    pats_p = torch.from_numpy(pats).pin_memory().numpy()
    off_p = torch.from_numpy(off.view(np.int64)).pin_memory().numpy().view(np.uint64)
    out = torch.zeros(npat, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    lat = np.zeros(first.size - 1)
    sv = capi.QFMServer(idx, slots=4)
    sv.replay(pats_p, off_p, first, np.zeros(first.size - 1), out, lat)
    st = sv.stats()
    sv.close()
    assert st["error"] == 0 and st["completed"] == first.size - 1
    assert st["mean_requests_per_batch"] > 1          # requests shared batches
    ids = np.array(g["sample_ids"], dtype=np.int64)
    want = np.array(g["sample_counts"], dtype=np.uint64)
    assert np.array_equal(out[ids], want), first_diff(out[ids], want)
    plain = torch.empty(npat, dtype=torch.int64, device="cuda")
    capi.qfm_count(idx, dev_u8(pats), dev_u64(off), plain)
    assert np.array_equal(out, host_u64(plain))
    assert (lat > 0).all()
    assert capi.qfm_status(idx) == 0
    idx.free()
