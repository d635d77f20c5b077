"""GPU parity of region-batched rank (qr_set_batch_mode QR_BATCH_REGIONS)
against the oracle, bit-exact.

Region batching sorts every tile of 8192 queries by text region (256
regions), answers the sorted runs region after region and puts the results
back in query order (rank_4 too, with its four counts per query).  The cases cover several tiles with a ragged last tile, every region,
out-of-range positions and symbols inside the batch, degenerate orders (all
queries equal, sorted, reversed, everything in the first or last region),
tiny texts where regions are single positions, batch sizes around the tile
size, the automatic rule, two streams at once, and agreement with the direct
kernels on a large batch.
"""
import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth
from tests.gpu_util import build, dev_u64, dev_u8, host_u64

pytestmark = pytest.mark.gpu

TILE = 8192
B2, S2, B4, S4 = 496, 496 * 128, 224, 224 * 256
# the paper, sector and inline layouts (the 128-byte line layout always runs direct);
# QR_LAYOUT_INLINE32X2 (4) is sigma 2 only, QR_LAYOUT_INLINE24_8 (5) sigma 4 only
LAYOUTS = [0, 1, 3, 4]
DNA_LAYOUTS = [0, 1, 3, 5]
U64MAX = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def regions_index(words, n, sigma, layout):
    from paper_2602_04103_gb300 import capi
    idx = build(words, n, sigma, layout)
    capi.qr_set_batch_mode(idx, capi.QR_BATCH_REGIONS)
    return idx


def run(idx, q, c):
    import torch
    from paper_2602_04103_gb300 import capi
    assert capi.qr_rank_plan(idx, q.size) == (capi.QR_BATCH_REGIONS if q.size else capi.QR_BATCH_DIRECT)
    dq = dev_u64(q)
    out = torch.empty_like(dq)
    if isinstance(c, (int, np.integer)):
        capi.qr_rank(idx, dq, int(c), out)
    else:
        capi.qr_rank_c(idx, dq, dev_u8(c), out)
    return host_u64(out)


def expect(words, n, sigma, q, c):
    """Oracle ranks, UINT64_MAX where q > n or the symbol is out of range."""
    c_arr = np.full(q.size, c, dtype=np.uint8) if isinstance(c, (int, np.integer)) else c
    ok = (q <= n) & (c_arr < sigma)
    want = np.full(q.size, U64MAX, dtype=np.uint64)
    if ok.any():
        w, rc = oracle.rank_c(words, n, sigma, q[ok], c_arr[ok])
        assert rc == 0
        want[ok] = w
    return want


def check(idx, words, n, sigma, q, c, status=0):
    from paper_2602_04103_gb300 import capi
    got = run(idx, q, c)
    want = expect(words, n, sigma, q, c)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (n, sigma, q.size, bad[:5], got[bad[:5]], want[bad[:5]])
    assert capi.qr_status(idx) == status


RANK_VARIANTS = range(4)   # qr_set_region_tuning


@pytest.mark.parametrize("variant", RANK_VARIANTS)
@pytest.mark.parametrize("tiles", [1, 38, 32])
def test_every_rank_pass_variant(variant, tiles):
    """Every rank-pass variant, on batches whose tile count is 1, not a
    multiple of the 16 runs of a step, and a multiple of it; every
    region-batched layout, both alphabets, bad queries and symbols inside."""
    from paper_2602_04103_gb300 import capi
    m = tiles * TILE - (123 if tiles > 1 else 0)
    n2, n4 = 7 * S2 + 11, 5 * S4 + 13
    words = synth.bits(synth.base_seed(70), n2, 0.5)
    dwords = synth.dna_uniform(synth.base_seed(71), n4)
    q2 = synth.queries(synth.base_seed(72) + tiles, n2, m)
    q2[::1009] = n2 + 3
    q4 = synth.queries(synth.base_seed(73) + tiles, n4, m)
    cv = synth.symbols(synth.base_seed(74) + tiles, m, 4)
    cv[::997] = 4
    for layout in sorted(set(LAYOUTS) | set(DNA_LAYOUTS)):
        if layout in LAYOUTS:
            idx = regions_index(words, n2, 2, layout)
            capi.qr_set_region_tuning(idx, variant)
            check(idx, words, n2, 2, q2, 1, status=capi.QR_ERANGE)
            idx.free()
        if layout in DNA_LAYOUTS:
            idx = regions_index(dwords, n4, 4, layout)
            capi.qr_set_region_tuning(idx, variant)
            check(idx, dwords, n4, 4, q4, cv, status=capi.QR_EBADSYM)
            idx.free()


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_region_length_rule_both_sides(layout):
    """The region length grows by one doubling when the doubled region holds
    at most 24 MiB of index per 2^28 queries of the batch: over this ~96 KB
    sigma-4 index a batch of 4096 queries keeps the plain shift and one of
    2^16 takes the doubled one.  Both give the oracle's results (rank with
    per-query symbols, rank_4), bad positions and symbols included."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 5 * S4 + 17
    words = synth.dna_uniform(synth.base_seed(80), n)
    idx = regions_index(words, n, 4, layout)
    for m in (4096, 1 << 16):
        q = synth.queries(synth.base_seed(81) + m, n, m)
        q[::733] = n + 1
        cv = synth.symbols(synth.base_seed(82) + m, m, 4)
        cv[::977] = 9
        check(idx, words, n, 4, q, cv, status=capi.QR_ERANGE | capi.QR_EBADSYM)
        ok = q <= n
        want4, rc = oracle.rank4(words, n, q[ok])
        dq = dev_u64(q)
        out4 = torch.empty((m, 4), dtype=torch.int64, device="cuda")
        capi.qr_rank4(idx, dq, out4)
        got4 = host_u64(out4).reshape(-1, 4)
        assert rc == 0 and np.array_equal(got4[ok], want4), m
        assert (got4[~ok] == U64MAX).all()
        assert capi.qr_status(idx) == capi.QR_ERANGE
    idx.free()


def test_region_tuning_range():
    from paper_2602_04103_gb300 import capi
    idx = build(synth.bits(1, 1000, 0.5), 1000, 2, 1)
    for v in (-1, 4):
        with pytest.raises(capi.QRError):
            capi.qr_set_region_tuning(idx, v)
    idx.free()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_bits_tiles_ragged(layout):
    n = 3 * S2 + 1234
    words = synth.bits(synth.base_seed(40), n, 0.5)
    idx = regions_index(words, n, 2, layout)
    m = 3 * TILE + 77
    q = synth.queries(synth.base_seed(41), n, m)
    for c in (0, 1):
        check(idx, words, n, 2, q, c)
    cv = synth.symbols(synth.base_seed(42), m, 2)
    check(idx, words, n, 2, q, cv)


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_dna_tiles_ragged(layout):
    n = 3 * S4 + 777
    words = synth.dna_gc_runs(synth.base_seed(43), n, 0.4, 0.05, 10, 1000)
    idx = regions_index(words, n, 4, layout)
    m = 2 * TILE + 4099
    q = synth.queries(synth.base_seed(44), n, m)
    for c in range(4):
        check(idx, words, n, 4, q, c)
    check(idx, words, n, 4, q, synth.symbols(synth.base_seed(45), m, 4))


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_prefix_rank_tiles_ragged(layout):
    """prefix_rank (the count of characters at most c before q) through
    region batching, against the oracle, with out-of-range positions."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 2 * S4 + 4321
    words = synth.dna_gc_runs(synth.base_seed(60), n, 0.4, 0.05, 10, 1000)
    idx = regions_index(words, n, 4, layout)
    m = 2 * TILE + 123
    q = synth.queries(synth.base_seed(61), n, m)
    q[::211] = n + 5
    ok = q <= n
    assert capi.qr_rank_plan(idx, m, 2) == capi.QR_BATCH_REGIONS
    dq = dev_u64(q)
    out = torch.empty_like(dq)
    for c in range(4):
        capi.qr_prefix_rank(idx, dq, c, out)
        got = host_u64(out)
        want, rc = oracle.prefix_rank(words, n, 4, q[ok], c)
        assert rc == 0 and np.array_equal(got[ok], want), (layout, c)
        assert (got[~ok] == U64MAX).all()
        assert capi.qr_status(idx) == capi.QR_ERANGE


@pytest.mark.parametrize("layout", sorted(set(LAYOUTS) | set(DNA_LAYOUTS)))
@pytest.mark.parametrize("sigma", [2, 4])
def test_bad_queries_inside_batch(layout, sigma):
    from paper_2602_04103_gb300 import capi
    if sigma == 4 and layout not in DNA_LAYOUTS:
        pytest.skip("BiRank32x2 is sigma 2 only")
    if sigma == 2 and layout not in LAYOUTS:
        pytest.skip("QuadRank24_8 is sigma 4 only")
    n = 2 * (S2 if sigma == 2 else S4) + 999
    words = synth.bits(7, n, 0.3) if sigma == 2 else synth.dna_uniform(8, n)
    idx = regions_index(words, n, sigma, layout)
    m = TILE + 500
    q = synth.queries(synth.base_seed(46), n, m)
    q[::97] = n + 1 + np.arange(q[::97].size, dtype=np.uint64)   # out of range
    q[5] = U64MAX
    q[6] = n                                                     # largest valid position
    check(idx, words, n, sigma, q, 1, status=capi.QR_ERANGE)
    cv = synth.symbols(synth.base_seed(47), m, sigma)
    cv[::89] = sigma                                             # bad symbols
    cv[3] = 255
    q2 = synth.queries(synth.base_seed(48), n, m)
    check(idx, words, n, sigma, q2, cv, status=capi.QR_EBADSYM)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("order", ["equal", "sorted", "reversed", "first_region", "last_region", "zero", "n"])
def test_degenerate_orders(layout, order):
    n = 5 * S2 + 17
    words = synth.bits(synth.base_seed(49), n, 0.5)
    idx = regions_index(words, n, 2, layout)
    m = 2 * TILE + 333
    q = synth.queries(synth.base_seed(50), n, m)
    if order == "equal":
        q[:] = q[0]
    elif order == "sorted":
        q.sort()
    elif order == "reversed":
        q = np.sort(q)[::-1].copy()
    elif order == "first_region":
        q = q % np.uint64(max(1, n >> 9))
    elif order == "last_region":
        q = np.uint64(n) - q % np.uint64(max(1, n >> 9))
    elif order == "zero":
        q[:] = 0
    else:
        q[:] = n
    check(idx, words, n, 2, q, 1)


@pytest.mark.parametrize("layout", sorted(set(LAYOUTS) | set(DNA_LAYOUTS)))
@pytest.mark.parametrize("n", [0, 1, 2, 255, 256, 257, 495, 496, 497, 1000])
def test_tiny_texts(layout, n):
    """Texts shorter than 256 regions: a region is one or a few positions."""
    q = np.concatenate([np.arange(n + 1, dtype=np.uint64), synth.queries(n + 12, n, 3000)])
    if layout in LAYOUTS:
        words = synth.bits(n + 11, n, 0.5)
        idx = regions_index(words, n, 2, layout)
        for c in (0, 1):
            check(idx, words, n, 2, q, c)
    if layout in DNA_LAYOUTS:
        dwords = synth.dna_uniform(n + 13, n)
        idx4 = regions_index(dwords, n, 4, layout)
        check(idx4, dwords, n, 4, q, synth.symbols(n + 14, q.size, 4))


@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 4095, 4096, 4097, TILE - 1, TILE, TILE + 1, 2 * TILE + 1])
def test_batch_sizes(m):
    n = 2 * S2 + 5
    words = synth.bits(synth.base_seed(51), n, 0.5)
    for layout in LAYOUTS:
        idx = regions_index(words, n, 2, layout)
        check(idx, words, n, 2, synth.queries(synth.base_seed(52) + m, n, m), 1)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_unaligned_query_array(layout):
    """Queries that start 8 bytes past a 16-byte boundary: the sort pass then
    reads them with plain loads instead of bulk copies; the results agree."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 3 * S2 + 99
    words = synth.bits(synth.base_seed(62), n, 0.5)
    idx = regions_index(words, n, 2, layout)
    m = 3 * TILE + 17
    q = synth.queries(synth.base_seed(63), n, m + 1)
    dq = dev_u64(q)[1:]                     # 8-byte aligned view
    assert dq.data_ptr() % 16 == 8
    out = torch.empty(m, dtype=torch.int64, device="cuda")
    capi.qr_rank(idx, dq, 1, out)
    assert np.array_equal(host_u64(out), expect(words, n, 2, q[1:], 1))
    assert capi.qr_status(idx) == 0


@pytest.mark.parametrize("layout", [1, 3])
@pytest.mark.parametrize("m", [TILE, 3 * TILE + 17])
def test_unaligned_output_array(layout, m):
    """Output arrays 16-byte aligned and 8 bytes past a 16-byte boundary agree
    with the oracle, on full and partial tiles, for rank and prefix_rank."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 3 * S2 + 99
    words = synth.bits(synth.base_seed(64), n, 0.5)
    idx = regions_index(words, n, 2, layout)
    q = synth.queries(synth.base_seed(65) + m, n, m)
    q[::501] = n + 7
    dq = dev_u64(q)
    for off in (0, 1):
        out = torch.empty(m + 1, dtype=torch.int64, device="cuda")[off:off + m]
        assert out.data_ptr() % 16 == 8 * off
        capi.qr_rank(idx, dq, 0, out)
        assert np.array_equal(host_u64(out), expect(words, n, 2, q, 0)), off
        assert capi.qr_status(idx) == capi.QR_ERANGE
    n4 = 2 * S4 + 5
    w4 = synth.dna_uniform(synth.base_seed(66), n4)
    idx4 = regions_index(w4, n4, 4, layout)
    q4 = synth.queries(synth.base_seed(67) + m, n4, m)
    dq4 = dev_u64(q4)
    for off in (0, 1):
        out = torch.empty(m + 1, dtype=torch.int64, device="cuda")[off:off + m]
        capi.qr_prefix_rank(idx4, dq4, 2, out)
        want, rc = oracle.prefix_rank(w4, n4, 4, q4, 2)
        assert rc == 0 and np.array_equal(host_u64(out), want), off


def test_empty_batch():
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1000
    idx = regions_index(synth.bits(3, n, 0.5), n, 2, 0)
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    capi.qr_rank(idx, empty, 1, empty)
    assert capi.qr_status(idx) == 0


def test_agrees_with_direct_large_batch():
    """2^22 queries over a 2^30-bit text (138 MB index, larger than half of L2):
    region batching and the direct kernels agree on every output, and a
    sample matches the oracle.  The automatic rule picks region batching here."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 30
    words = synth.bits(synth.base_seed(53), n, 0.5)
    q = synth.queries(synth.base_seed(54), n, 1 << 22)
    dq = dev_u64(q)
    for layout in LAYOUTS:
        idx = build(words, n, 2, layout)
        assert capi.qr_rank_plan(idx, q.size) == capi.QR_BATCH_REGIONS
        assert capi.qr_rank_plan(idx, 1 << 16) == capi.QR_BATCH_DIRECT
        a, b = torch.empty_like(dq), torch.empty_like(dq)
        capi.qr_rank(idx, dq, 1, a)                      # automatic: regions
        capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT)
        assert capi.qr_rank_plan(idx, q.size) == capi.QR_BATCH_DIRECT
        capi.qr_rank(idx, dq, 1, b)
        assert torch.equal(a, b), layout
        sample = np.arange(0, q.size, 997)
        want, rc = oracle.rank(words, n, 2, q[sample], 1)
        assert rc == 0 and np.array_equal(host_u64(a)[sample], want)
        assert capi.qr_status(idx) == 0
        idx.free()


@pytest.mark.parametrize("order", ["sorted", "equal", "half_sorted"])
def test_auto_clustered_batches(order):
    """Under the automatic rule a device probe sends clustered batches to the
    direct kernels (and the region passes return at once); the outputs are
    the same whichever path runs."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 30
    words = synth.bits(synth.base_seed(58), n, 0.5)
    q = synth.queries(synth.base_seed(59), n, 1 << 22)
    if order == "sorted":
        q.sort()
    elif order == "equal":
        q[:] = q[7]
    else:
        q[: q.size // 2].sort()
    dq = dev_u64(q)
    for layout in LAYOUTS:
        idx = build(words, n, 2, layout)
        assert capi.qr_rank_plan(idx, q.size) == capi.QR_BATCH_REGIONS
        a, b = torch.empty_like(dq), torch.empty_like(dq)
        capi.qr_rank(idx, dq, 0, a)
        capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT)
        capi.qr_rank(idx, dq, 0, b)
        assert torch.equal(a, b), (order, layout)
        sample = np.arange(0, q.size, 1009)
        want, rc = oracle.rank(words, n, 2, q[sample], 0)
        assert rc == 0 and np.array_equal(host_u64(a)[sample], want)
        assert capi.qr_status(idx) == 0
        idx.free()


def test_auto_rule_small_index_stays_direct():
    from paper_2602_04103_gb300 import capi
    n = 1 << 24   # 2.2 MB index: L2-resident
    idx = build(synth.bits(5, n, 0.5), n, 2, 0)
    assert capi.qr_rank_plan(idx, 1 << 26) == capi.QR_BATCH_DIRECT
    assert capi.qr_rank_plan(idx, 1 << 26, 1) == capi.QR_BATCH_DIRECT
    capi.qr_set_batch_mode(idx, capi.QR_BATCH_REGIONS)
    assert capi.qr_rank_plan(idx, 1 << 26) == capi.QR_BATCH_REGIONS
    assert capi.qr_rank_plan(idx, 1 << 26, 1) == capi.QR_BATCH_DIRECT   # rank_4 is sigma 4 only
    idx4 = build(synth.dna_uniform(6, n), n, 4, 1)
    capi.qr_set_batch_mode(idx4, capi.QR_BATCH_REGIONS)
    assert capi.qr_rank_plan(idx4, 1 << 26, 1) == capi.QR_BATCH_REGIONS
    assert capi.qr_rank_plan(idx4, 1 << 26, 2) == capi.QR_BATCH_REGIONS
    idx128 = build(synth.bits(5, n, 0.5), n, 2, 2)
    capi.qr_set_batch_mode(idx128, capi.QR_BATCH_REGIONS)
    assert capi.qr_rank_plan(idx128, 1 << 26) == capi.QR_BATCH_DIRECT   # 128-byte lines always direct
    with pytest.raises(capi.QRError):
        capi.qr_set_batch_mode(idx, 7)


def test_two_streams_and_timing():
    """Region-batched calls on two streams at once (each with its own pooled
    scratch), then the per-pass timing aid."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 4 * S2 + 3
    words = synth.bits(synth.base_seed(55), n, 0.5)
    idx = regions_index(words, n, 2, 0)
    qa = synth.queries(synth.base_seed(56), n, 5 * TILE + 1)
    qb = synth.queries(synth.base_seed(57), n, 3 * TILE + 9)
    dqa, dqb = dev_u64(qa), dev_u64(qb)
    oa, ob = torch.empty_like(dqa), torch.empty_like(dqb)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        capi.qr_rank(idx, dqa, 1, oa, stream=sa)
        capi.qr_rank(idx, dqb, 0, ob, stream=sb)
    torch.cuda.synchronize()
    assert np.array_equal(host_u64(oa), expect(words, n, 2, qa, 1))
    assert np.array_equal(host_u64(ob), expect(words, n, 2, qb, 0))
    capi.qr_region_timing(idx, True)
    capi.qr_rank(idx, dqa, 1, oa)
    ms = capi.qr_region_timing(idx, False, read=True)
    assert len(ms) == 3 and all(x >= 0 for x in ms)
    assert np.array_equal(host_u64(oa), expect(words, n, 2, qa, 1))
    capi.qr_release_scratch()
    capi.qr_rank(idx, dqa, 1, oa)                     # the pool refills after a release
    assert np.array_equal(host_u64(oa), expect(words, n, 2, qa, 1))
    assert capi.qr_status(idx) == 0


def test_sort_wait_runs_out_and_reports_timeout():
    """Failure path without a GPU fault: the test hook withholds one bulk copy
    of the sort pass, so its bounded wait (0.25 s) runs out.  The call reports
    QR_ETIMEOUT, its other passes return at once, and the next call on the
    same context is correct."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 3 * S2 + 7
    words = synth.bits(synth.base_seed(64), n, 0.5)
    idx = regions_index(words, n, 2, 1)
    m = 4 * TILE                                # whole tiles: the sort pass moves them by bulk copies
    q = synth.queries(synth.base_seed(65), n, m)
    dq = dev_u64(q)
    out = torch.full((m,), -7, dtype=torch.int64, device="cuda")
    capi.qr_set_region_fault(idx, True)
    capi.qr_rank(idx, dq, 1, out)
    assert capi.qr_status(idx) == capi.QR_ETIMEOUT
    assert (out == -7).all()                    # the unsort pass returned without writing
    capi.qr_set_region_fault(idx, False)
    capi.qr_rank(idx, dq, 1, out)
    assert np.array_equal(host_u64(out), expect(words, n, 2, q, 1))
    assert capi.qr_status(idx) == 0


def rank4_regions(idx, q):
    """qr_rank4 through region batching."""
    import torch
    from paper_2602_04103_gb300 import capi
    assert capi.qr_rank_plan(idx, q.size, 1) == (capi.QR_BATCH_REGIONS if q.size else capi.QR_BATCH_DIRECT)
    dq = dev_u64(q)
    out = torch.full((q.size, 4), -7, dtype=torch.int64, device="cuda")
    capi.qr_rank4(idx, dq, out)
    return host_u64(out).reshape(-1, 4)


def expect4(words, n, q):
    ok = q <= n
    want = np.full((q.size, 4), U64MAX, dtype=np.uint64)
    if ok.any():
        w, rc = oracle.rank4(words, n, q[ok])
        assert rc == 0
        want[ok] = w
    return want


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_rank4_tiles_ragged(layout):
    """rank_4 through region batching: every query's row of four counts;
    out-of-range positions give rows of UINT64_MAX and QR_ERANGE.  An output
    not 16-byte aligned is refused."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 3 * S4 + 777
    words = synth.dna_gc_runs(synth.base_seed(70), n, 0.4, 0.05, 10, 1000)
    idx = regions_index(words, n, 4, layout)
    m = 2 * TILE + 4099
    q = synth.queries(synth.base_seed(71), n, m)
    got = rank4_regions(idx, q)
    assert np.array_equal(got, expect4(words, n, q))
    assert capi.qr_status(idx) == 0
    q[::101] = n + 3
    q[7] = U64MAX
    q[8] = n
    got = rank4_regions(idx, q)
    assert np.array_equal(got, expect4(words, n, q))
    assert capi.qr_status(idx) == capi.QR_ERANGE
    flat = torch.full((4 * m + 2,), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.QRError):
        capi.qr_rank4(idx, dev_u64(q), flat[1:-1].view(m, 4))
    # 16 bytes past a 32-byte boundary: rows written as two 16-byte stores
    out = flat[2:].view(m, 4)
    assert out.data_ptr() % 32 == 16
    capi.qr_rank4(idx, dev_u64(q), out)
    assert np.array_equal(host_u64(out).reshape(-1, 4), expect4(words, n, q))
    assert capi.qr_status(idx) == capi.QR_ERANGE


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
@pytest.mark.parametrize("order", ["equal", "sorted", "reversed", "last_region", "zero"])
def test_rank4_degenerate_orders_and_unaligned_queries(layout, order):
    import torch
    from paper_2602_04103_gb300 import capi
    n = 4 * S4 + 31
    words = synth.dna_uniform(synth.base_seed(72), n)
    idx = regions_index(words, n, 4, layout)
    m = 2 * TILE + 5
    q = synth.queries(synth.base_seed(73), n, m)
    if order == "equal":
        q[:] = q[0]
    elif order == "sorted":
        q.sort()
    elif order == "reversed":
        q = np.sort(q)[::-1].copy()
    elif order == "last_region":
        q = np.uint64(n) - q % np.uint64(max(1, n >> 9))
    else:
        q[:] = 0
    assert np.array_equal(rank4_regions(idx, q), expect4(words, n, q))
    # queries 8 bytes past a 16-byte boundary: the plain sort pass
    qq = np.concatenate([[np.uint64(0)], q]).astype(np.uint64)
    dq = dev_u64(qq)[1:]
    assert dq.data_ptr() % 16 == 8
    out = torch.empty((m, 4), dtype=torch.int64, device="cuda")
    capi.qr_rank4(idx, dq, out)
    assert np.array_equal(host_u64(out).reshape(-1, 4), expect4(words, n, q))
    assert capi.qr_status(idx) == 0


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
@pytest.mark.parametrize("n", [0, 1, 2, 223, 224, 225, 255, 256, 1000])
def test_rank4_tiny_texts_and_sizes(layout, n):
    words = synth.dna_uniform(n + 21, n)
    idx = regions_index(words, n, 4, layout)
    q = np.concatenate([np.arange(n + 1, dtype=np.uint64), synth.queries(n + 22, n, 3000)])
    assert np.array_equal(rank4_regions(idx, q), expect4(words, n, q))
    for m in (1, 31, TILE - 1, TILE + 1):
        qm = synth.queries(n + 23 + m, n, m)
        assert np.array_equal(rank4_regions(idx, qm), expect4(words, n, qm))


def test_rank4_agrees_with_direct_large_batch():
    """2^22 rank_4 queries over 2^29 chars (a 153-179 MB index, larger than
    half of L2, with more than two queries per 128 bytes of it): the
    automatic rule takes region batching, and it agrees with the direct
    kernels on every output; a sample matches the oracle."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 29
    words = synth.dna_uniform(synth.base_seed(74), n)
    q = synth.queries(synth.base_seed(75), n, 1 << 22)
    dq = dev_u64(q)
    for layout in DNA_LAYOUTS:
        idx = build(words, n, 4, layout)
        assert capi.qr_rank_plan(idx, q.size, 1) == capi.QR_BATCH_REGIONS
        a = torch.empty((q.size, 4), dtype=torch.int64, device="cuda")
        b = torch.empty_like(a)
        capi.qr_rank4(idx, dq, a)
        capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT)
        capi.qr_rank4(idx, dq, b)
        assert torch.equal(a, b), layout
        sample = np.arange(0, q.size, 991)
        want, rc = oracle.rank4(words, n, q[sample])
        assert rc == 0 and np.array_equal(host_u64(a).reshape(-1, 4)[sample], want)
        assert capi.qr_status(idx) == 0
        idx.free()


def test_region_rank4_timeout_leaves_output_untouched():
    """The sort pass's bounded wait running out (test hook) stops the rank_4
    passes too: QR_ETIMEOUT, the output untouched, the next call right."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 3 * S4 + 7
    words = synth.dna_uniform(synth.base_seed(76), n)
    idx = regions_index(words, n, 4, 1)
    m = 4 * TILE
    q = synth.queries(synth.base_seed(77), n, m)
    dq = dev_u64(q)
    out = torch.full((m, 4), -7, dtype=torch.int64, device="cuda")
    capi.qr_set_region_fault(idx, True)
    capi.qr_rank4(idx, dq, out)
    assert capi.qr_status(idx) == capi.QR_ETIMEOUT
    assert (out == -7).all()
    capi.qr_set_region_fault(idx, False)
    capi.qr_rank4(idx, dq, out)
    assert np.array_equal(host_u64(out).reshape(-1, 4), expect4(words, n, q))
    assert capi.qr_status(idx) == 0
