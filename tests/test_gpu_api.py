"""The object methods of the binding against the oracle: QRIndex.rank
(scalar and per-query symbols), rank4 and prefix_rank, and QFMIndex.count
(one strand and both).  Each method allocates its output on the queries'
device and calls the C-ABI entry point of the same name."""
import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth
from tests.gpu_util import dev_u64, dev_u8, host_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def test_qrindex_methods_bits():
    from paper_2602_04103_gb300 import capi
    n = 3 * 496 * 128 + 11                      # three superblocks and a ragged tail
    words = synth.bits(synth.base_seed(80), n, 0.5)
    q = synth.queries(synth.base_seed(81), n, 5000)
    idx = capi.qr_build(dev_u64(words), n, 2)
    dq = dev_u64(q)
    for c in (0, 1):
        want, rc = oracle.rank(words, n, 2, q, c)
        assert rc == 0
        assert np.array_equal(host_u64(idx.rank(dq, c)), want)
    assert idx.status() == 0
    idx.free()
    assert idx.handle is None


def test_qrindex_methods_dna():
    from paper_2602_04103_gb300 import capi
    n = 2 * 224 * 256 + 5
    text = synth.dna_uniform(synth.base_seed(82), n)
    q = synth.queries(synth.base_seed(83), n, 5000)
    cs = synth.symbols(synth.base_seed(84), q.size, 4)
    idx = capi.qr_build(dev_u64(text), n, 4)
    dq = dev_u64(q)
    want, rc = oracle.rank_c(text, n, 4, q, cs)
    assert rc == 0
    assert np.array_equal(host_u64(idx.rank(dq, dev_u8(cs))), want)
    want4, rc = oracle.rank4(text, n, q)
    assert rc == 0
    got4 = idx.rank4(dq)
    assert tuple(got4.shape) == (q.size, 4)
    assert np.array_equal(host_u64(got4).reshape(-1, 4), want4)
    wantp, rc = oracle.prefix_rank(text, n, 4, q, 2)
    assert rc == 0
    assert np.array_equal(host_u64(idx.prefix_rank(dq, 2)), wantp)
    assert idx.status() == 0


def test_qfmindex_count_one_and_both_strands():
    from paper_2602_04103_gb300 import capi
    t = synth.fm_text(85, 1 << 16, repeat_cover=0.2, len_min=300, len_max=2000, sub_rate=0.02)
    idx = capi.qfm_build(dev_u8(t), t.size)
    pats, off = synth.patterns(86, t, 5000, 1, 150, sub_rate=0.01)
    m = off.size - 1
    sa = oracle.suffix_array(t)
    dp, doff = dev_u8(pats), dev_u64(off)
    both = host_u64(idx.count(dp, doff, capi.QFM_BOTH_STRANDS))
    assert both.size == 2 * m
    assert np.array_equal(both[:m], oracle.count_sa(t, sa, pats, off))
    assert np.array_equal(both[m:], oracle.count_sa(t, sa, oracle.revcomp_batch(pats, off), off))
    assert np.array_equal(host_u64(idx.count(dp, doff)), both[:m])
    assert idx.status() == 0
