"""Continuous-batching server: every request's counts are the same whether it
runs alone (one qfm_count call on its own patterns) or packed with other
requests into shared batches, in every server mode; admission limits and a
batch failure injected on the host are reported, not hung."""
import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth
from tests.gpu_util import dev_u64, dev_u8, host_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    from paper_2602_04103_gb300 import capi
    torch.cuda.set_device(0)
    n = 1 << 20
    text = synth.fm_text(201, n, repeat_cover=0.2, len_min=300, len_max=3000, sub_rate=0.02)
    idx = capi.qfm_build(dev_u8(text), n)
    yield text, idx
    idx.free()


def make_requests(text, nreq, seed, max_m=300):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, max_m + 1, nreq)
    pats, off = synth.patterns(seed, text, int(sizes.sum()), 16, 250, 0.01)
    first = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    return pats, off, first


def alone(idx, pats, off, first):
    """Counts of each request computed by its own qfm_count call."""
    import torch
    from paper_2602_04103_gb300 import capi
    res = np.empty(off.size - 1, np.uint64)
    for r in range(first.size - 1):
        a, b = int(first[r]), int(first[r + 1])
        sub_off = (off[a:b + 1] - off[a]).astype(np.uint64)
        o = torch.empty(b - a, dtype=torch.int64, device="cuda")
        capi.qfm_count(idx, dev_u8(pats[off[a]:off[b]]), dev_u64(sub_off), o)
        res[a:b] = host_u64(o)
    return res


def pinned(a: np.ndarray) -> np.ndarray:
    """A page-locked copy of a, as a numpy view of a pinned torch tensor."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t.numpy()


@pytest.mark.parametrize("mode", ["batched", "per_request", "small_slots", "pinned_direct", "pinned_per_request",
                                  "stream_calls", "pinned_stream_calls"])
def test_mixed_equals_alone(fm, mode):
    from paper_2602_04103_gb300 import capi
    text, idx = fm
    pats, off, first = make_requests(text, 200, 7)
    want = alone(idx, pats, off, first)
    opts = {"batched": dict(slots=4), "per_request": dict(slots=1, max_requests_per_batch=1),
            "small_slots": dict(slots=3, max_batch_patterns=700, max_batch_bytes=700 * 250),
            "pinned_direct": dict(slots=4), "pinned_per_request": dict(slots=1, max_requests_per_batch=1),
            "stream_calls": dict(slots=4, use_graph=0), "pinned_stream_calls": dict(slots=4, use_graph=0)}[mode]
    sv = capi.QFMServer(idx, **opts)
    if mode.startswith("pinned"):
        # back-to-back requests in page-locked buffers: batches copy straight from them
        pats, off = pinned(pats), pinned(off)
        out = pinned(np.full(off.size - 1, np.uint64(2 ** 64 - 1)))
    else:
        out = np.full(off.size - 1, np.uint64(2 ** 64 - 1))
    offs = []
    for r in range(first.size - 1):
        a, b = int(first[r]), int(first[r + 1])
        offs.append(off[a:b + 1] if mode.startswith("pinned") else np.ascontiguousarray(off[a:b + 1]))
        sv.submit(pats, offs[-1], out[a:b])
    sv.drain(120)
    ids, lat, st = sv.poll(1000)
    assert ids.size == 200 and (st == 0).all() and (lat > 0).all()
    assert np.array_equal(out, want)
    stats = sv.stats()
    assert stats["completed"] == 200 and stats["error"] == 0
    # each batch is one launch of the slot's CUDA graph unless graphs are off
    if "stream_calls" in mode:
        assert stats["graph_batches"] == 0
    else:
        assert stats["graph_batches"] == stats["batches"]
    if mode == "per_request":
        assert stats["mean_requests_per_batch"] == 1.0
    sv.close()
    # and the counts are the oracle's
    sample = np.arange(0, off.size - 1, 53)
    sub = np.concatenate([pats[off[k]:off[k + 1]] for k in sample])
    sub_off = np.concatenate([[0], np.cumsum((off[sample + 1] - off[sample]).astype(np.int64))]).astype(np.uint64)
    assert np.array_equal(out[sample], oracle.count_brute_batch(text, sub, sub_off))


@pytest.mark.parametrize("pin", [False, True])
def test_replay_poisson_trace(fm, pin):
    from paper_2602_04103_gb300 import capi
    text, idx = fm
    pats, off, first = make_requests(text, 300, 11)
    want = alone(idx, pats, off, first)
    if pin:
        pats, off = pinned(pats), pinned(off)
    rng = np.random.default_rng(3)
    arrival = np.cumsum(rng.exponential(1e-4, 300))
    for opts in (dict(slots=4), dict(slots=1, max_requests_per_batch=1)):
        sv = capi.QFMServer(idx, **opts)
        out = pinned(np.zeros(off.size - 1, np.uint64)) if pin else np.zeros(off.size - 1, np.uint64)
        lat = np.zeros(300)
        mk = sv.replay(pats, off, first, arrival, out, lat)
        assert np.array_equal(out, want)
        assert (lat > 0).all() and mk >= arrival[-1]
        sv.close()


def test_admission_limits_and_injected_failure(fm):
    from paper_2602_04103_gb300 import capi
    text, idx = fm
    with pytest.raises(capi.QRError):      # slots x capacity above the budget
        capi.QFMServer(idx, budget_bytes=1 << 20, slots=4, max_batch_bytes=1 << 20)
    sv = capi.QFMServer(idx, slots=2, max_batch_patterns=100, max_batch_bytes=100 * 250)
    pats, off, first = make_requests(text, 1, 5, max_m=300)
    big = np.ascontiguousarray(off)
    if big.size - 1 > 100:
        with pytest.raises(capi.QRError):  # a request larger than a batch slot
            sv.submit(pats, big, np.zeros(big.size - 1, np.uint64))
    with pytest.raises(capi.QRError):      # offsets[m] < offsets[0]
        sv.submit(pats, np.array([5, 3], np.uint64), np.zeros(1, np.uint64))
    # offsets out of order inside a request: that pattern counts 0 and sets the status bit
    pats2 = np.zeros(64, np.uint8)
    out2 = np.full(2, np.uint64(7))
    sv.submit(pats2, np.array([0, 40, 20], np.uint64), out2)
    sv.drain(30)
    assert out2[0] == 0
    assert capi.qfm_status(idx) == capi.QR_EBADSYM
    sv.close()
    # batches after the second fail on the host: their requests report the error
    sv = capi.QFMServer(idx, slots=1, max_requests_per_batch=1, fail_after_batches=2)
    pats, off, first = make_requests(text, 6, 9, max_m=50)
    outs = []
    for r in range(6):
        a, b = int(first[r]), int(first[r + 1])
        outs.append(np.zeros(b - a, np.uint64))
        sv.submit(pats, np.ascontiguousarray(off[a:b + 1]), outs[-1])
    with pytest.raises(capi.QRError) as e:
        sv.drain(60)
    assert e.value.code == capi.QR_ECUDA and "injected" in str(e.value)
    ids, lat, st = sv.poll(100)
    assert ids.size == 6
    assert (st[np.argsort(ids)][:2] == 0).all() and (st[np.argsort(ids)][2:] == capi.QR_ECUDA).all()
    assert sv.stats()["error"] == capi.QR_ECUDA
    sv.close()
