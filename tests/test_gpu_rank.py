"""GPU parity of BiRank / QuadRank rank, rank with per-query symbols and
rank_4 against the oracle: bit-exact (integer results).

Covers tiny exhaustive texts, multi-superblock texts with every q, edge
lengths around block and superblock boundaries, adversarial texts that reach
the largest 16-bit deltas the paper's bounds allow (Sec. 3: b_j <= S + 2^11 - 1;
Sec. 4: S4 + 2^13 - 1), out-of-range queries and symbols, every launch
tuning, the host-buffer pipeline and the layout itself.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth
from tests.gpu_util import build, dev_u64, dev_u8, host_u64, rank, rank4

pytestmark = pytest.mark.gpu

B2, S2, B4, S4 = 496, 496 * 128, 224, 224 * 256
B2S, S2S, B4S, S4S = 480, 480 * 128, 192, 192 * 256
B2L, S2L, B4L, S4L = 1008, 1008 * 32, 480, 480 * 64
B2W, B2X, B4W, L0 = 480, 448, 192, 1 << 22   # inline-32 layouts: data per line, lines per L0 entry
L0_24 = 1 << 16                                # QuadRank24_8: lines per L0 entry
# QR_LAYOUT_PAPER (BiRank16 / QuadRank16), _SECTOR, _LINE128, _INLINE32 (BiRank32 /
# QuadRank32), _INLINE32X2 (BiRank32x2, sigma 2 only), _INLINE24_8 (QuadRank24_8,
# sigma 4 only)
BI_LAYOUTS = [0, 1, 2, 3, 4]
DNA_LAYOUTS = [0, 1, 2, 3, 5]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def check_bits(words, n, q=None, cs=(0, 1), layout=0):
    idx = build(words, n, 2, layout)
    q = np.arange(n + 1, dtype=np.uint64) if q is None else q
    for c in cs:
        want, rc = oracle.rank(words, n, 2, q, c)
        assert rc == 0
        got = rank(idx, q, c)
        assert np.array_equal(got, want), (n, c, np.flatnonzero(got != want)[:5])
    return idx


def check_dna(words, n, q=None, layout=0):
    idx = build(words, n, 4, layout)
    q = np.arange(n + 1, dtype=np.uint64) if q is None else q
    w4, rc = oracle.rank4(words, n, q)
    assert rc == 0
    assert np.array_equal(rank4(idx, q), w4), n
    for c in range(4):
        assert np.array_equal(rank(idx, q, c), w4[:, c]), (n, c)
    cv = synth.symbols(n + 17, q.size, 4)
    assert np.array_equal(rank(idx, q, cv), w4[np.arange(q.size), cv])
    return idx


@pytest.mark.parametrize("layout", BI_LAYOUTS)
def test_tiny_exhaustive_bits(layout):
    for L in range(0, 11):
        for bits in itertools.product([0, 1], repeat=L):
            check_bits(synth.pack_bits(np.array(bits, dtype=np.uint8)), L, layout=layout)


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_tiny_exhaustive_dna(layout):
    for L in range(0, 6):
        for codes in itertools.product(range(4), repeat=L):
            check_dna(synth.pack2(np.array(codes, dtype=np.uint8)), L, layout=layout)


@pytest.mark.parametrize("layout", BI_LAYOUTS)
@pytest.mark.parametrize("p", [0.5, 0.01, 0.99])
def test_multi_superblock_bits_every_q(p, layout):
    n = 3 * S2 + 1234
    words = synth.bits(synth.base_seed(1) + int(p * 100), n, p)
    check_bits(words, n, layout=layout)


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
@pytest.mark.parametrize("kind", ["uniform", "gc_runs"])
def test_multi_superblock_dna_every_q(kind, layout):
    n = 3 * S4 + 777
    words = synth.dna_uniform(5, n) if kind == "uniform" else synth.dna_gc_runs(6, n, 0.4, 0.05, 10, 1000)
    check_dna(words, n, layout=layout)


@pytest.mark.parametrize("n", [0, 1, 63, 64, 111, 112, 113, 119, 120, 121, 223, 224, 225, 239, 240, 241, 255, 256,
                               335, 336, 337, 359, 360, 361, 447, 448, 449, 479, 480, 481, 495, 496, 497, 503,
                               504, 505, 895, 896, 897, 991, 992, 993, 1007, 1008, 1009, 2016,
                               S2L - 1, S2L, S2L + 1, S2S - 1, S2S, S2S + 1, S2 - 1, S2, S2 + 1,
                               2 * S2, 2 * S2 + 240])
def test_edge_lengths_bits(n):
    for layout in BI_LAYOUTS:
        check_bits(synth.bits(n + 3, n, 0.5), n, layout=layout)


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 47, 48, 49, 63, 64, 65, 95, 96, 97, 127, 128, 129, 143, 144, 145,
                               191, 192, 193, 255, 256, 257, 319, 320, 321,
                               223, 224, 225, 239, 240, 241, 447, 448, 449, 479, 480, 481, S4L - 1, S4L, S4L + 1,
                               S4S - 1, S4S, S4S + 1, S4 - 1, S4, S4 + 1, 2 * S4 + 96])
def test_edge_lengths_dna(n):
    for layout in DNA_LAYOUTS:
        check_dna(synth.dna_uniform(n + 5, n), n, layout=layout)


def read_layout(idx, sigma):
    import torch
    from paper_2602_04103_gb300 import capi
    info = capi.qr_info(idx)
    lines = np.empty(info["bytes_blocks"] // 8, dtype=np.uint64)
    sup = np.empty(info["bytes_super"] // 4, dtype=np.uint32)
    capi.qr_copy_layout(idx, lines, sup)
    return info, lines.reshape(-1, 8), sup


def test_max_delta_bits():
    # superblock 0 holds 2047 ones then zeros, so rank(S) mod 2^11 = 2047; superblock
    # 1 is all ones: its last block's delta is 2047 + 127 * 496 + 240 = 65279
    n = 2 * S2 + 3000
    bits = np.zeros(n, dtype=np.uint8)
    bits[:2047] = 1
    bits[S2:2 * S2] = 1
    words = synth.pack_bits(bits)
    idx = check_bits(words, n)
    info, lines, sup = read_layout(idx, 2)
    deltas = (lines[:, 0] & np.uint64(0xFFFF)).astype(np.int64)
    assert deltas.max() == 2047 + 127 * B2 + 240 == 65279
    assert sup.tolist()[:3] == [0, 0, (2047 + S2) >> 11]


def test_max_delta_dna():
    n = 2 * S4 + 5000
    codes = np.zeros(n, dtype=np.uint8)
    codes[:8191] = 3
    codes[S4:2 * S4] = 3
    words = synth.pack2(codes)
    idx = check_dna(words, n, q=np.concatenate([np.arange(0, n + 1, 7), [n]]).astype(np.uint64))
    info, lines, sup = read_layout(idx, 4)
    d3 = ((lines[:, 1] >> np.uint64(16)) & np.uint64(0xFFFF)).astype(np.int64)   # b_{j,T}
    assert d3.max() == 8191 + 255 * B4 + 96 == 65407


def test_layout_matches_definitions():
    # b_j = rank(jB + 240) - 2^11 s_{j/128}, s_i = floor(rank(iS) / 2^11)   (Sec. 3)
    n = 4 * S2 + 4321
    words = synth.bits(99, n, 0.37)
    idx = build(words, n, 2)
    info, lines, sup = read_layout(idx, 2)
    nb = n // B2 + 1
    assert info["nblocks"] == nb and lines.shape[0] == nb
    js = np.arange(nb, dtype=np.uint64)
    mids = np.minimum(js * np.uint64(B2) + np.uint64(240), np.uint64(n))
    r_mid, _ = oracle.rank(words, n, 2, mids, 1)
    # past the end the text is padded with zeros, so rank(min(x, n)) is the padded rank
    starts = np.arange(info["nsuper"], dtype=np.uint64) * np.uint64(S2)
    r_sup, _ = oracle.rank(words, n, 2, np.minimum(starts, np.uint64(n)), 1)
    assert np.array_equal(sup.astype(np.uint64), r_sup >> np.uint64(11))
    want_b = r_mid - (sup.astype(np.uint64)[js >> np.uint64(7)] << np.uint64(11))
    assert np.array_equal(lines[:, 0] & np.uint64(0xFFFF), want_b)
    # the data bits follow the delta: line bit 16 + d = text bit jB + d
    tb = np.unpackbits(words.view(np.uint8), bitorder="little")
    lb = np.unpackbits(lines.view(np.uint8), bitorder="little").reshape(nb, 512)
    for j in [0, 1, 127, 128, nb - 1]:
        lo, hi = j * B2, min(j * B2 + B2, n)
        assert np.array_equal(lb[j, 16:16 + hi - lo], tb[lo:hi])
        assert lb[j, 16 + hi - lo:].sum() == 0


def test_layout_matches_definitions_dna():
    # b_{j,c} = rank(jB4 + 96, c) - 2^13 s_{j/256,c}; transposed, negated data (Sec. 4)
    n = 2 * S4 + 999
    words = synth.dna_uniform(123, n)
    idx = build(words, n, 4)
    info, lines, sup = read_layout(idx, 4)
    sup = sup.reshape(-1, 4).astype(np.uint64)
    nb = info["nblocks"]
    js = np.arange(nb, dtype=np.uint64)
    mids = np.minimum(js * np.uint64(B4) + np.uint64(96), np.uint64(n))
    r4, _ = oracle.rank4(words, n, mids)
    # padding chars are A (code 0): the padded rank of A at a middle past n grows by the excess
    excess = (js * np.uint64(B4) + np.uint64(96)) - mids
    r4[:, 0] += excess
    starts = np.minimum(np.arange(info["nsuper"], dtype=np.uint64) * np.uint64(S4), np.uint64(n))
    rs, _ = oracle.rank4(words, n, starts)
    assert np.array_equal(sup, rs >> np.uint64(13))
    w0, w1 = lines[:, 0], lines[:, 1]
    got = np.stack([w0 & np.uint64(0xFFFF), (w0 >> np.uint64(16)) & np.uint64(0xFFFF),
                    w1 & np.uint64(0xFFFF), (w1 >> np.uint64(16)) & np.uint64(0xFFFF)], axis=1)
    assert np.array_equal(got, r4 - (sup[js >> np.uint64(8)] << np.uint64(13)))
    # slot s of the line holds data char s - 32: raw low bit = ~word[4h+2g] bit
    codes = synth.unpack2(words, n)
    for j in [0, 1, 255, 256, nb - 1]:
        for slot in range(32, 256):
            d = j * B4 + slot - 32
            h, g, b = slot // 128, (slot % 128) // 64, slot % 64
            lo = (~int(lines[j, 4 * h + 2 * g]) >> b) & 1
            hi = (~int(lines[j, 4 * h + 2 * g + 1]) >> b) & 1
            want = int(codes[d]) if d < n else 0
            assert lo | (hi << 1) == want, (j, slot)


def test_sizes_and_paper_overheads():
    from paper_2602_04103_gb300 import capi
    for n in [1 << 20, 3 * S2 + 5]:
        idx = build(synth.bits(1, n, 0.5), n, 2)
        info = capi.qr_info(idx)
        nb = n // B2 + 1
        assert info["bytes_blocks"] == 64 * nb
        assert info["bytes_super"] == 4 * ((nb + 127) // 128)
    # overheads from the closed forms at large n: 3.28% (Sec. 3) and 14.40% (Sec. 4)
    n2 = 1 << 34
    nb = n2 // B2 + 1
    over2 = (64 * nb + 4 * ((nb + 127) // 128)) * 8 / n2 - 1
    assert abs(over2 * 100 - 3.28) < 0.005
    n4 = 1 << 32
    nb4 = n4 // B4 + 1
    over4 = (64 * nb4 + 16 * ((nb4 + 255) // 256)) * 8 / (2 * n4) - 1
    assert abs(over4 * 100 - 14.40) < 0.005


def test_out_of_range_and_bad_symbols():
    from paper_2602_04103_gb300 import capi
    n = S2 + 10
    words = synth.bits(3, n, 0.5)
    idx = build(words, n, 2)
    q = np.array([0, n, n + 1, 1 << 40, 5], dtype=np.uint64)
    got = rank(idx, q, 1)
    want, _ = oracle.rank(words, n, 2, np.array([0, n, 5], dtype=np.uint64), 1)
    assert got[[0, 1, 4]].tolist() == want.tolist()
    assert got[2] == np.uint64(2 ** 64 - 1) and got[3] == np.uint64(2 ** 64 - 1)
    assert capi.qr_status(idx) == capi.QR_ERANGE
    assert capi.qr_status(idx) == 0
    got = rank(idx, np.array([1, 2, 3], dtype=np.uint64), np.array([1, 2, 0], dtype=np.uint8))
    assert got[1] == np.uint64(2 ** 64 - 1)
    assert capi.qr_status(idx) == capi.QR_EBADSYM
    with pytest.raises(capi.QRError):
        rank(idx, q, 2)
    n4 = 1000
    w4 = synth.dna_uniform(4, n4)
    idx4 = build(w4, n4, 4)
    r = rank4(idx4, np.array([n4 + 1, 3], dtype=np.uint64))
    assert (r[0] == np.uint64(2 ** 64 - 1)).all()
    assert capi.qr_status(idx4) == capi.QR_ERANGE
    with pytest.raises(capi.QRError):
        rank4(idx, np.array([1], dtype=np.uint64))   # sigma 2 index


@pytest.mark.parametrize("k", [1, 2, 4, 8])
@pytest.mark.parametrize("load,layout", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (0, 1), (0, 2), (0, 3), (0, 4),
                                         (0, 5)])
@pytest.mark.parametrize("threads", [64, 256, 512])
def test_every_tuning(k, load, layout, threads):
    from paper_2602_04103_gb300 import capi
    if layout == 2 and k > 2:
        pytest.skip("the 128-byte line layout takes 1 or 2 queries per thread")
    n, n4 = 3 * S2 + 77, 3 * S4 + 99
    words, w4 = synth.bits(17, n, 0.5), synth.dna_uniform(18, n4)
    q = synth.queries(19, n, 100_003)
    q4 = synth.queries(20, n4, 100_003)
    cv = synth.symbols(21, q4.size, 4)
    idx = build(words, n, 2, layout if layout in BI_LAYOUTS else 0)
    capi.qr_set_tuning(idx, k, threads, load, 0)
    assert np.array_equal(rank(idx, q, 1), oracle.rank(words, n, 2, q, 1)[0])
    if layout in DNA_LAYOUTS:
        idx4 = build(w4, n4, 4, layout)
        capi.qr_set_tuning(idx4, k, threads, load, 0)
        assert np.array_equal(rank(idx4, q4, cv), oracle.rank_c(w4, n4, 4, q4, cv)[0])
        assert np.array_equal(rank4(idx4, q4), oracle.rank4(w4, n4, q4)[0])
    capi.qr_set_tuning(idx, k, threads, load, 7)    # explicit small grid: grid-stride loop
    assert np.array_equal(rank(idx, q, 0), oracle.rank(words, n, 2, q, 0)[0])


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_host_pipeline_matches_device(layout):
    import torch
    from paper_2602_04103_gb300 import capi
    n = 5 * S4 + 3
    w4 = synth.dna_uniform(31, n)
    idx = build(w4, n, 4, layout)
    m = (1 << 23) * 4 + 12345                   # more chunks than streams, ragged
    q = synth.queries(32, n, m)
    cv = synth.symbols(33, m, 4)
    qh = torch.from_numpy(q.view(np.int64)).pin_memory()
    ch = torch.from_numpy(cv).pin_memory()
    out = torch.empty(m, dtype=torch.int64).pin_memory()
    capi.qr_rank_host(idx, qh, ch, out)
    want1, _ = oracle.rank_c(w4, n, 4, q, cv)
    assert np.array_equal(out.numpy().view(np.uint64), want1)
    out4 = torch.empty((m, 4), dtype=torch.int64).pin_memory()
    capi.qr_rank4_host(idx, qh, out4)
    want4, _ = oracle.rank4(w4, n, q)
    assert np.array_equal(out4.numpy().view(np.uint64), want4)
    capi.qr_rank_host(idx, qh, 2, out)
    assert np.array_equal(out.numpy().view(np.uint64), want4[:, 2])
    # pageable host memory works too
    outp = np.empty(m, dtype=np.uint64)
    capi.qr_rank_host(idx, q, 1, outp)
    assert np.array_equal(outp, want4[:, 1])


def test_concurrent_streams_same_index():
    import torch
    from paper_2602_04103_gb300 import capi
    n = 2 * S2 + 5
    words = synth.bits(41, n, 0.5)
    idx = build(words, n, 2)
    streams = [torch.cuda.Stream() for _ in range(4)]
    qs = [synth.queries(50 + i, n, 200_000) for i in range(4)]
    outs = []
    for s, q in zip(streams, qs):
        with torch.cuda.stream(s):
            dq = dev_u64(q)
            o = torch.empty_like(dq)
            capi.qr_rank(idx, dq, 1, o, stream=s)
            outs.append((dq, o))
    torch.cuda.synchronize()
    for (dq, o), q in zip(outs, qs):
        assert np.array_equal(host_u64(o), oracle.rank(words, n, 2, q, 1)[0])


def test_sector_layout_matches_definitions():
    # BiRank16x2 (Sec. 3.1): deltas to 1/4 and 3/4 of a 480-bit block,
    # b_{j,h} = rank(480 j + 240 h + 120) - 2^11 s_{j/128}; half h holds data
    # bits [480 j + 240 h, +240) after its 16-bit delta
    from paper_2602_04103_gb300 import capi
    n = 4 * S2S + 4321
    words = synth.bits(77, n, 0.41)
    idx = build(words, n, 2, 1)
    info, lines, sup = read_layout(idx, 2)
    nb = n // B2S + 1
    assert info["nblocks"] == nb and info["block_chars"] == 480
    starts = np.minimum(np.arange(info["nsuper"], dtype=np.uint64) * np.uint64(S2S), np.uint64(n))
    r_sup, _ = oracle.rank(words, n, 2, starts, 1)
    assert np.array_equal(sup.astype(np.uint64), r_sup >> np.uint64(11))
    js = np.arange(nb, dtype=np.uint64)
    tb = np.unpackbits(words.view(np.uint8), bitorder="little")
    lb = np.unpackbits(lines.view(np.uint8), bitorder="little").reshape(nb, 2, 256)
    for h in range(2):
        mids = np.minimum(js * np.uint64(B2S) + np.uint64(240 * h + 120), np.uint64(n))
        r_mid, _ = oracle.rank(words, n, 2, mids, 1)
        want = r_mid - (sup.astype(np.uint64)[js >> np.uint64(7)] << np.uint64(11))
        assert np.array_equal(lines[:, 4 * h] & np.uint64(0xFFFF), want)
        for j in [0, 1, 127, 128, nb - 1]:
            lo, hi = j * B2S + 240 * h, min(j * B2S + 240 * h + 240, n)
            if hi > lo:
                assert np.array_equal(lb[j, h, 16:16 + hi - lo], tb[lo:hi])


def test_sector_max_deltas():
    # sigma 2: 2047 + 127 * 480 + 240 + 120 = 63367; sigma 4: 8191 + 255 * 192 + 96 + 48 = 57295
    n = 2 * S2S + 3000
    bits = np.zeros(n, dtype=np.uint8)
    bits[:2047] = 1
    bits[S2S:2 * S2S] = 1
    idx = check_bits(synth.pack_bits(bits), n, layout=1)
    _, lines, _ = read_layout(idx, 2)
    d = np.maximum(lines[:, 0] & np.uint64(0xFFFF), lines[:, 4] & np.uint64(0xFFFF)).astype(np.int64)
    assert d.max() == 63367
    n4 = 2 * S4S + 5000
    codes = np.zeros(n4, dtype=np.uint8)
    codes[:8191] = 3
    codes[S4S:2 * S4S] = 3
    idx4 = check_dna(synth.pack2(codes), n4, q=np.concatenate([np.arange(0, n4 + 1, 7), [n4]]).astype(np.uint64),
                     layout=1)
    _, lines4, _ = read_layout(idx4, 4)
    dT = np.maximum(lines4[:, 0] >> np.uint64(48), lines4[:, 4] >> np.uint64(48)).astype(np.int64)
    assert dT.max() == 57295


def test_sector_sizes_and_overheads():
    from paper_2602_04103_gb300 import capi
    n = 3 * S2S + 5
    info = capi.qr_info(build(synth.bits(1, n, 0.5), n, 2, 1))
    nb = n // 480 + 1
    assert info["bytes_blocks"] == 64 * nb and info["bytes_super"] == 4 * ((nb + 127) // 128)
    # BiRank16x2's overhead as printed in Sec. 3.1: 6.72%
    n2 = 1 << 34
    nb = n2 // 480 + 1
    over = (64 * nb + 4 * ((nb + 127) // 128)) * 8 / n2 - 1
    assert abs(over * 100 - 6.72) < 0.005


def test_autotune_and_build_tuned():
    import torch
    from paper_2602_04103_gb300 import capi
    n = 6 * S2 + 5
    words = synth.bits(61, n, 0.5)
    q = synth.queries(62, n, 300_000)
    dq = dev_u64(q)
    scratch = torch.empty_like(dq)
    idx = build(words, n, 2, 0)
    t = capi.qr_autotune(idx, dq, scratch, c=1)
    assert t["queries_per_thread"] in (1, 2, 4, 8) and t["load_mode"] in (0, 1, 2, 3, 4)
    assert capi.qr_get_tuning(idx) == t
    assert np.array_equal(rank(idx, q, 1), oracle.rank(words, n, 2, q, 1)[0])
    # a 5% space budget admits only BiRank16 (3.28%); 7% admits BiRank16x2 (6.72%)
    # and BiRank32 (6.67%) too, and the fastest of the three on this batch wins
    idx5, lay5 = capi.qr_build_tuned(dev_u64(words), n, 2, dq, scratch, c=1, max_overhead=0.05)
    assert lay5 == 0
    idx7, lay7 = capi.qr_build_tuned(dev_u64(words), n, 2, dq, scratch, c=0, max_overhead=0.07)
    assert lay7 in (0, 1, 3)
    for i in (idx5, idx7):
        assert np.array_equal(rank(i, q, 0), oracle.rank(words, n, 2, q, 0)[0])
    with pytest.raises(capi.QRError):
        capi.qr_build_tuned(dev_u64(words), n, 2, dq, scratch, max_overhead=0.01)
    n4 = 3 * S4 + 1
    w4 = synth.dna_uniform(63, n4)
    q4 = synth.queries(64, n4, 100_000)
    dq4 = dev_u64(q4)
    s4 = torch.empty((q4.size, 4), dtype=torch.int64, device="cuda")
    idx4, lay4 = capi.qr_build_tuned(dev_u64(w4), n4, 4, dq4, s4, rank4=True, max_overhead=0.40)
    assert np.array_equal(rank4(idx4, q4), oracle.rank4(w4, n4, q4)[0])


def test_line128_layout_matches_definitions():
    # sigma 2: delta to data offset 504 of a 1008-bit block, 32 lines per superblock
    n = 3 * S2L + 777
    words = synth.bits(88, n, 0.45)
    idx = build(words, n, 2, 2)
    from paper_2602_04103_gb300 import capi
    info = capi.qr_info(idx)
    assert info["line_bytes"] == 128 and info["block_chars"] == 1008 and info["super_blocks"] == 32
    lines = np.empty(info["bytes_blocks"] // 8, dtype=np.uint64)
    sup = np.empty(info["bytes_super"] // 4, dtype=np.uint32)
    capi.qr_copy_layout(idx, lines, sup)
    lines = lines.reshape(-1, 16)
    nb = n // B2L + 1
    js = np.arange(nb, dtype=np.uint64)
    starts = np.minimum(np.arange(info["nsuper"], dtype=np.uint64) * np.uint64(S2L), np.uint64(n))
    assert np.array_equal(sup.astype(np.uint64), oracle.rank(words, n, 2, starts, 1)[0] >> np.uint64(11))
    mids = np.minimum(js * np.uint64(B2L) + np.uint64(504), np.uint64(n))
    want = oracle.rank(words, n, 2, mids, 1)[0] - (sup.astype(np.uint64)[js >> np.uint64(5)] << np.uint64(11))
    assert np.array_equal(lines[:, 0] & np.uint64(0xFFFF), want)
    tb = np.unpackbits(words.view(np.uint8), bitorder="little")
    lb = np.unpackbits(lines.view(np.uint8), bitorder="little").reshape(nb, 1024)
    for j in [0, 1, 31, 32, nb - 1]:
        lo, hi = j * B2L, min(j * B2L + B2L, n)
        assert np.array_equal(lb[j, 16:16 + hi - lo], tb[lo:hi])
    # sigma 4: chars 64g.. in words 2+2g (~low) / 3+2g (~high), tail 448..479 in word 1
    n4 = 2 * S4L + 333
    w4 = synth.dna_uniform(89, n4)
    idx4 = build(w4, n4, 4, 2)
    info4 = capi.qr_info(idx4)
    l4 = np.empty(info4["bytes_blocks"] // 8, dtype=np.uint64)
    s4 = np.empty(info4["bytes_super"] // 4, dtype=np.uint32)
    capi.qr_copy_layout(idx4, l4, s4)
    l4 = l4.reshape(-1, 16)
    s4 = s4.reshape(-1, 4).astype(np.uint64)
    nb4 = info4["nblocks"]
    js = np.arange(nb4, dtype=np.uint64)
    mids = np.minimum(js * np.uint64(B4L) + np.uint64(240), np.uint64(n4))
    r4 = oracle.rank4(w4, n4, mids)[0]
    r4[:, 0] += (js * np.uint64(B4L) + np.uint64(240)) - mids     # padding chars are A
    got = np.stack([(l4[:, 0] >> np.uint64(16 * c)) & np.uint64(0xFFFF) for c in range(4)], axis=1)
    assert np.array_equal(got, r4 - (s4[js >> np.uint64(6)] << np.uint64(13)))
    codes = synth.unpack2(w4, n4)
    for j in [0, 63, 64, nb4 - 1]:
        for d in range(480):
            i = j * B4L + d
            if d < 448:
                g, b = d // 64, d % 64
                lo = (~int(l4[j, 2 + 2 * g]) >> b) & 1
                hi = (~int(l4[j, 3 + 2 * g]) >> b) & 1
            else:
                b = d - 448
                lo = (~int(l4[j, 1]) >> b) & 1
                hi = (~int(l4[j, 1]) >> (32 + b)) & 1
            assert lo | (hi << 1) == (int(codes[i]) if i < n4 else 0), (j, d)


def test_line128_max_deltas_and_overheads():
    # sigma 2: 2047 + 31 * 1008 + 504 = 33799; sigma 4: 8191 + 63 * 480 + 240 = 38671
    n = 2 * S2L + 3000
    bits = np.zeros(n, dtype=np.uint8)
    bits[:2047] = 1
    bits[S2L:2 * S2L] = 1
    idx = check_bits(synth.pack_bits(bits), n, layout=2)
    from paper_2602_04103_gb300 import capi
    info = capi.qr_info(idx)
    lines = np.empty(info["bytes_blocks"] // 8, dtype=np.uint64)
    capi.qr_copy_layout(idx, lines, None)
    assert int((lines.reshape(-1, 16)[:, 0] & np.uint64(0xFFFF)).max()) == 33799
    n4 = 2 * S4L + 5000
    codes = np.zeros(n4, dtype=np.uint8)
    codes[:8191] = 3
    codes[S4L:2 * S4L] = 3
    idx4 = check_dna(synth.pack2(codes), n4, q=np.concatenate([np.arange(0, n4 + 1, 5), [n4]]).astype(np.uint64),
                     layout=2)
    info4 = capi.qr_info(idx4)
    l4 = np.empty(info4["bytes_blocks"] // 8, dtype=np.uint64)
    capi.qr_copy_layout(idx4, l4, None)
    assert int((l4.reshape(-1, 16)[:, 0] >> np.uint64(48)).max()) == 38671
    # overheads at large n (closed forms): 1.69% and 6.88%
    n2 = 1 << 34
    nb = n2 // 1008 + 1
    assert abs(((128 * nb + 4 * ((nb + 31) // 32)) * 8 / n2 - 1) * 100 - 1.69) < 0.005
    n4b = 1 << 32
    nb4 = n4b // 480 + 1
    assert abs(((128 * nb4 + 16 * ((nb4 + 63) // 64)) * 8 / (2 * n4b) - 1) * 100 - 6.88) < 0.01
    with pytest.raises(capi.QRError):
        capi.qr_set_tuning(idx, 4, 256, 0, 0)


@pytest.mark.parametrize("layout", DNA_LAYOUTS)
def test_prefix_rank(layout):
    import torch
    from paper_2602_04103_gb300 import capi
    n = 3 * S4 + 321
    w4 = synth.dna_gc_runs(71, n, 0.4, 0.05, 10, 1000)
    idx = build(w4, n, 4, layout)
    q = np.concatenate([synth.queries(72, n, 200_000), [0, n, n + 1]]).astype(np.uint64)
    dq = dev_u64(q)
    out = torch.empty_like(dq)
    for c in range(4):
        capi.qr_prefix_rank(idx, dq, c, out)
        want, rc = oracle.prefix_rank(w4, n, 4, q, c)
        assert rc == oracle.OR_ERANGE and np.array_equal(host_u64(out), want), c
    assert capi.qr_status(idx) == capi.QR_ERANGE
    with pytest.raises(capi.QRError):
        capi.qr_prefix_rank(idx, dq, 4, out)
    with pytest.raises(capi.QRError):
        capi.qr_prefix_rank(build(synth.bits(1, 100, 0.5), 100, 2), dq, 0, out)


@pytest.mark.parametrize("layout", sorted(set(BI_LAYOUTS) | set(DNA_LAYOUTS)))
@pytest.mark.parametrize("sigma", [2, 4])
def test_rank_chain(layout, sigma):
    import torch
    from paper_2602_04103_gb300 import capi
    if sigma == 4 and layout not in DNA_LAYOUTS:
        pytest.skip("BiRank32x2 is sigma 2 only")
    if sigma == 2 and layout not in BI_LAYOUTS:
        pytest.skip("QuadRank24_8 is sigma 4 only")
    n = 4 * S2 + 99 if sigma == 2 else 4 * S4 + 99
    words = synth.bits(91, n, 0.5) if sigma == 2 else synth.dna_uniform(92, n)
    idx = build(words, n, sigma, layout)
    q0 = np.concatenate([synth.queries(93, n, 5000), [0, n, n + 1]]).astype(np.uint64)
    out = torch.empty((q0.size, 2), dtype=torch.int64, device="cuda")
    for c in range(sigma):
        capi.qr_rank_chain(idx, dev_u64(q0), 50, c, out)
        want, rc = oracle.rank_chain(words, n, sigma, q0, 50, c)
        assert rc == oracle.OR_ERANGE
        assert np.array_equal(host_u64(out).reshape(-1, 2), want), c
    assert capi.qr_status(idx) == capi.QR_ERANGE
    with pytest.raises(capi.QRError):
        capi.qr_rank_chain(idx, dev_u64(q0), 0, 0, out)
    # one chain alone (a warp with a single live lane) and a single step
    one = torch.empty((1, 2), dtype=torch.int64, device="cuda")
    capi.qr_rank_chain(idx, dev_u64(q0[:1]), 1, sigma - 1, one)
    want, _ = oracle.rank_chain(words, n, sigma, q0[:1], 1, sigma - 1)
    assert np.array_equal(host_u64(one).reshape(-1, 2), want)


@pytest.mark.parametrize("nbytes,load_bytes,k", [(32, 16, 4), (32, 32, 4), (64, 32, 2), (128, 32, 1),
                                                 (128, 128, 1), (128, 128, 2)])
def test_probe_gather_digests(nbytes, load_bytes, k):
    """The measurement probe reads whole records: every digest is the XOR of
    the 64-bit words of one record (also for the quad-cooperative 128-byte
    reads), and a ragged last tile is written without running past m."""
    import torch
    from paper_2602_04103_gb300 import capi
    nrec, m = 1000, 5003
    words = synth.bits(synth.base_seed(60), nrec * nbytes * 8, 0.5)[: nrec * nbytes // 8]
    buf = torch.from_numpy(words.view(np.int64)).cuda()
    out = torch.full((m + 64,), -1, dtype=torch.int64, device="cuda")
    capi.qr_probe_gather(buf, nrec, nbytes, m, 7, out, k, 256, load_bytes=load_bytes)
    torch.cuda.synchronize()
    rec = words.reshape(nrec, nbytes // 8)
    digests = set(int(x) for x in np.bitwise_xor.reduce(rec, axis=1))
    got = out.cpu().numpy().view(np.uint64)
    assert all(int(x) in digests for x in got[:m])
    assert (got[m:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    assert len(set(got[:m].tolist())) > nrec // 2      # many distinct records drawn


def test_probe_gather_rejects_quad_mode_on_small_records():
    import torch
    from paper_2602_04103_gb300 import capi
    buf = torch.zeros(1024, dtype=torch.int64, device="cuda")
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError):
        capi.qr_probe_gather(buf, 128, 64, 16, 7, out, 1, 256, load_bytes=128)


def test_small_configuration_every_output():
    """The small BiRank configuration: n = 2^24 i.i.d. bits (p = 0.5), 10^6
    uniform queries in [0, n]; every output of every layout and of the tuned
    build, both symbols, against the oracle's linear prefix sweep."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    n = 1 << 24
    words = synth.bits(synth.base_seed(1), n, 0.5)
    q = synth.queries(synth.substream(synth.base_seed(1), 2), n, 10 ** 6)
    want1, rc = oracle.rank(words, n, 2, q, 1)
    assert rc == 0
    want0 = q - want1
    dq = dev_u64(q)
    out = torch.empty_like(dq)
    for layout in BI_LAYOUTS:
        idx = build(words, n, 2, layout)
        for c, want in ((1, want1), (0, want0)):
            capi.qr_rank(idx, dq, c, out)
            assert np.array_equal(host_u64(out), want), (layout, c)
        assert capi.qr_status(idx) == 0
        idx.free()
    idx, layout, _ = workloads.build_tuned(dev_u64(words), n, 2, dq, c=1)
    capi.qr_rank(idx, dq, 1, out)
    assert np.array_equal(host_u64(out), want1), layout
    idx.free()


# ---------------------------------------------------------------- 32-bit inline layouts
def read_inline(idx):
    """(info, lines as uint64 words [nb, 8], L0 table as uint64)."""
    from paper_2602_04103_gb300 import capi
    info = capi.qr_info(idx)
    lines = np.empty(info["bytes_blocks"] // 8, dtype=np.uint64)
    l0 = np.empty(info["bytes_super"] // 8, dtype=np.uint64)
    capi.qr_copy_layout(idx, lines, l0)
    return info, lines.reshape(-1, 8), l0


@pytest.mark.parametrize("layout", [3, 4])
def test_inline_layout_matches_definitions_bits(layout):
    """BiRank32 (Sec. 3.1): one 32-bit value per line = rank(480 j + 240) minus
    the rank at the start of the line's L0 block (2^22 lines), data bit d at
    line bit 32 + d.  BiRank32x2: per 32-byte half h, the value = rank(448 j +
    224 h + 112) minus the same L0 rank, data bit d of the half at half bit
    32 + d.  The L0 table holds rank(L0 block start)."""
    n = 9 * S2 + 4321
    words = synth.bits(199, n, 0.37)
    idx = build(words, n, 2, layout)
    info, lines, l0 = read_inline(idx)
    per = B2W if layout == 3 else B2X
    nb = n // per + 1
    assert info["nblocks"] == nb and info["super_blocks"] == L0 and info["nsuper"] == 1
    assert l0.tolist() == [0]                       # one L0 block: rank 0 at its start
    js = np.arange(nb, dtype=np.uint64)
    tb = np.unpackbits(words.view(np.uint8), bitorder="little")
    lb = np.unpackbits(lines.view(np.uint8), bitorder="little").reshape(nb, 512)
    if layout == 3:
        mids = np.minimum(js * np.uint64(B2W) + np.uint64(240), np.uint64(n))
        r_mid, _ = oracle.rank(words, n, 2, mids, 1)   # padding bits are 0
        assert np.array_equal(lines[:, 0] & np.uint64(0xFFFFFFFF), r_mid)
        for j in [0, 1, 2, nb - 1]:
            lo, hi = j * B2W, min(j * B2W + B2W, n)
            assert np.array_equal(lb[j, 32:32 + hi - lo], tb[lo:hi])
            assert lb[j, 32 + hi - lo:].sum() == 0
    else:
        for h in (0, 1):
            mids = np.minimum(js * np.uint64(B2X) + np.uint64(224 * h + 112), np.uint64(n))
            r_mid, _ = oracle.rank(words, n, 2, mids, 1)
            assert np.array_equal(lines[:, 4 * h] & np.uint64(0xFFFFFFFF), r_mid), h
        for j in [0, 1, 2, nb - 1]:
            for h in (0, 1):
                lo, hi = j * B2X + 224 * h, min(j * B2X + 224 * h + 224, n)
                if hi <= lo:
                    assert lb[j, 256 * h + 32:256 * h + 256].sum() == 0
                    continue
                assert np.array_equal(lb[j, 256 * h + 32:256 * h + 32 + hi - lo], tb[lo:hi])
                assert lb[j, 256 * h + 32 + hi - lo:256 * h + 256].sum() == 0


def test_inline_layout_matches_definitions_dna():
    """QuadRank32 (Sec. 4.1): four 32-bit values per line, v_c = rank(192 j + 96,
    c) minus the L0 rank of c (word 0 = v0 | v1 << 32, word 1 = v2 | v3 << 32);
    words 2 + 2g / 3 + 2g = ~low / ~high bits of chars 64 g .. 64 g + 63."""
    n = 7 * S4 + 999
    words = synth.dna_uniform(223, n)
    idx = build(words, n, 4, 3)
    info, lines, l0 = read_inline(idx)
    nb = n // B4W + 1
    assert info["nblocks"] == nb and l0.tolist() == [0, 0, 0, 0]
    js = np.arange(nb, dtype=np.uint64)
    mids = np.minimum(js * np.uint64(B4W) + np.uint64(96), np.uint64(n))
    r4, _ = oracle.rank4(words, n, mids)
    r4[:, 0] += (js * np.uint64(B4W) + np.uint64(96)) - mids     # padding chars are A (code 0)
    w0, w1 = lines[:, 0], lines[:, 1]
    got = np.stack([w0 & np.uint64(0xFFFFFFFF), w0 >> np.uint64(32), w1 & np.uint64(0xFFFFFFFF),
                    w1 >> np.uint64(32)], axis=1)
    assert np.array_equal(got, r4)
    codes = synth.unpack2(words, n)
    for j in [0, 1, 2, nb - 1]:
        for d in range(B4W):
            g, b = d // 64, d % 64
            lo = (~int(lines[j, 2 + 2 * g]) >> b) & 1
            hi = (~int(lines[j, 3 + 2 * g]) >> b) & 1
            c = j * B4W + d
            assert lo | (hi << 1) == (int(codes[c]) if c < n else 0), (j, d)


def quad24_fields(lines):
    """QuadRank24_8's per-symbol words (word 0 = w0 | w1 << 32, word 1 = w2 |
    w3 << 32) split into a (low 24 bits) and b (high 8 bits), [nb, 4] each."""
    w0, w1 = lines[:, 0], lines[:, 1]
    w = np.stack([w0 & np.uint64(0xFFFFFFFF), w0 >> np.uint64(32), w1 & np.uint64(0xFFFFFFFF),
                  w1 >> np.uint64(32)], axis=1)
    return w & np.uint64(0xFFFFFF), w >> np.uint64(24)


def test_quad24_layout_matches_definitions():
    """QuadRank24_8 (Sec. 4.1): chars of QuadRank32 (words 2 + 2g / 3 + 2g =
    ~low / ~high bits of chars 64 g .. 64 g + 63); per symbol c,
    a_c = rank(192 j + 64, c) minus the rank of c at the start of the line's
    L0 block (2^16 lines) and b_c = the count of c in chars 64 .. 191 of the
    line, so that a_c + b_c = rank(192 j + 192, c) minus the same.  The text
    spans four L0 blocks, and the L0 table holds the rank at each start."""
    n = 3 * L0_24 * B4W + 5 * B4W + 77
    words = synth.dna_uniform(227, n)
    idx = build(words, n, 4, 5)
    info, lines, l0 = read_inline(idx)
    nb = n // B4W + 1
    assert info["nblocks"] == nb and info["super_blocks"] == L0_24 and info["nsuper"] == 4
    js = np.arange(nb, dtype=np.uint64)
    starts = np.minimum(np.arange(4, dtype=np.uint64) * np.uint64(L0_24 * B4W), np.uint64(n))
    want_l0, rc = oracle.rank4(words, n, starts, threads=4)
    assert rc == 0 and np.array_equal(l0.reshape(4, 4), want_l0)
    base = want_l0[(js // np.uint64(L0_24)).astype(np.int64)]
    a, b = quad24_fields(lines)
    for off, got in ((64, a), (192, a + b)):
        pos = js * np.uint64(B4W) + np.uint64(off)
        r4, rc = oracle.rank4(words, n, np.minimum(pos, np.uint64(n)), threads=4)
        r4[:, 0] += pos - np.minimum(pos, np.uint64(n))              # padding chars are A (code 0)
        assert rc == 0 and np.array_equal(got, r4 - base), off
    assert int(b.max()) <= 128 and int(a.max()) < L0_24 * B4W
    codes = synth.unpack2(words, n)
    for j in [0, 1, L0_24 - 1, L0_24, nb - 1]:
        for d in range(B4W):
            g, k = d // 64, d % 64
            lo = (~int(lines[j, 2 + 2 * g]) >> k) & 1
            hi = (~int(lines[j, 3 + 2 * g]) >> k) & 1
            c = j * B4W + d
            assert lo | (hi << 1) == (int(codes[c]) if c < n else 0), (j, d)


def test_quad24_l0_boundaries():
    """QuadRank24_8 over four L0 blocks: every query within 700 positions of
    each block start and of each group boundary of the lines there, plus
    2^20 uniform ones, against the oracle (rank with per-query symbols and
    rank_4), direct and region-batched."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 4 * L0_24 * B4W - 3
    words = synth.dna_gc_runs(synth.base_seed(305), n, 0.45, 0.05, 10, 2000)
    idx = build(words, n, 4, 5)
    starts = np.arange(1, 4) * (L0_24 * B4W)
    edges = np.concatenate([np.arange(b - 700, b + 700) for b in starts])
    q = np.concatenate([edges, synth.queries(synth.base_seed(306), n, 1 << 20), [0, n - 1, n]]).astype(np.uint64)
    want4, rc = oracle.rank4(words, n, q, threads=8)
    assert rc == 0
    cv = synth.symbols(synth.base_seed(307), q.size, 4)
    dq = dev_u64(q)
    for mode in (capi.QR_BATCH_DIRECT, capi.QR_BATCH_REGIONS):
        capi.qr_set_batch_mode(idx, mode)
        out4 = torch.empty((q.size, 4), dtype=torch.int64, device="cuda")
        capi.qr_rank4(idx, dq, out4)
        assert np.array_equal(host_u64(out4).reshape(-1, 4), want4), mode
        out = torch.empty_like(dq)
        capi.qr_rank_c(idx, dq, dev_u8(cv), out)
        assert np.array_equal(host_u64(out), want4[np.arange(q.size), cv]), mode
    assert capi.qr_status(idx) == 0
    idx.free()


def test_quad24_values_near_their_bound():
    """An all-T text over a whole L0 block: the last line's a_T reaches
    (2^16 - 1) * 192 + 64, the largest a 24-bit value holds here, and every
    b_T is 128; ranks around the next block's start are q for T, 0 for the
    rest."""
    n = L0_24 * B4W + 3000
    codes = np.full(n, 3, dtype=np.uint8)
    words = synth.pack2(codes)
    idx = build(words, n, 4, 5)
    info, lines, l0 = read_inline(idx)
    a, b = quad24_fields(lines)
    assert l0.reshape(-1, 4).tolist() == [[0, 0, 0, 0], [0, 0, 0, L0_24 * B4W]]
    assert int(a[L0_24 - 1, 3]) == (L0_24 - 1) * B4W + 64 < 1 << 24
    full = n // B4W                                            # lines before the partial last one
    assert (b[:full, 3] == 128).all() and (b[:full, :3] == 0).all()
    q = np.concatenate([np.arange(L0_24 * B4W - 1000, L0_24 * B4W + 1000), [n]]).astype(np.uint64)
    r4 = rank4(idx, q)
    assert np.array_equal(r4[:, 3], q) and not r4[:, :3].any()
    idx.free()


@pytest.mark.slow
@pytest.mark.parametrize("layout,sigma", [(3, 2), (4, 2), (3, 4)])
def test_inline_l0_blocks(layout, sigma):
    """Texts spanning several L0 blocks (2^22 lines each: 2^33 bits for
    BiRank32 / BiRank32x2, 2^31 chars for QuadRank32): the L0 table against
    the oracle's rank at every block start, and every query within 600
    positions of each block boundary plus 2^20 uniform ones against the
    oracle (rank, rank_4, both symbols), direct and region-batched."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 33 if sigma == 2 else 1 << 31
    words = synth.bits(synth.base_seed(301), n, 0.5) if sigma == 2 else synth.dna_uniform(synth.base_seed(302), n)
    per = {(3, 2): B2W, (4, 2): B2X, (3, 4): B4W}[(layout, sigma)]
    idx = build(words, n, sigma, layout)
    info, _, l0 = read_inline(idx)
    nl0 = (n // per + 1 + L0 - 1) // L0
    assert info["nsuper"] == nl0 >= 3
    starts = np.minimum(np.arange(nl0, dtype=np.uint64) * np.uint64(L0 * per), np.uint64(n))
    if sigma == 2:
        want_l0, _ = oracle.rank(words, n, 2, starts, 1)
        assert np.array_equal(l0, want_l0)
    else:
        want_l0, _ = oracle.rank4(words, n, starts)
        assert np.array_equal(l0.reshape(-1, 4), want_l0)
    edges = np.concatenate([np.arange(int(b) - 600, int(b) + 600) for b in starts[1:]])
    q = np.concatenate([edges, synth.queries(synth.base_seed(303), n, 1 << 20), [0, n]]).astype(np.uint64)
    dq = dev_u64(q)
    for mode in (capi.QR_BATCH_DIRECT, capi.QR_BATCH_REGIONS):
        capi.qr_set_batch_mode(idx, mode)
        if sigma == 2:
            out = torch.empty_like(dq)
            for c in (0, 1):
                capi.qr_rank(idx, dq, c, out)
                want, rc = oracle.rank(words, n, 2, q, c)
                assert rc == 0 and np.array_equal(host_u64(out), want), (mode, c)
        else:
            out4 = torch.empty((q.size, 4), dtype=torch.int64, device="cuda")
            capi.qr_rank4(idx, dq, out4)
            want4, rc = oracle.rank4(words, n, q)
            assert rc == 0 and np.array_equal(host_u64(out4).reshape(-1, 4), want4), mode
            cv = synth.symbols(synth.base_seed(304), q.size, 4)
            out = torch.empty_like(dq)
            capi.qr_rank_c(idx, dq, dev_u8(cv), out)
            assert np.array_equal(host_u64(out), want4[np.arange(q.size), cv]), mode
    assert capi.qr_status(idx) == 0
    idx.free()


@pytest.mark.slow
def test_inline_values_near_their_bound():
    """An all-ones text over a whole L0 block: the last lines' values reach
    2^22 * 448 - 112 (BiRank32x2), the largest a 32-bit value holds here."""
    n = L0 * B2X + 5000
    words = np.full((n + 63) // 64 + 1, np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    words[n // 64] = np.uint64((1 << (n % 64)) - 1)            # no bits at or beyond n
    words[n // 64 + 1:] = 0
    idx = build(words, n, 2, 4)
    info, lines, l0 = read_inline(idx)
    assert l0.tolist() == [0, L0 * B2X]
    assert int(lines[L0 - 1, 4] & np.uint64(0xFFFFFFFF)) == L0 * B2X - 112
    q = np.concatenate([np.arange(L0 * B2X - 1000, L0 * B2X + 1000), [n]]).astype(np.uint64)
    got = rank(idx, q, 1)
    assert np.array_equal(got, q)                              # rank of all ones is q
    assert np.array_equal(rank(idx, q, 0), np.zeros(q.size, dtype=np.uint64))
    idx.free()


def test_inline_sizes_and_overheads():
    """Overheads from the closed forms: BiRank32 6.67%, BiRank32x2 14.3%
    (Sec. 3.1), QuadRank32 33.3% (Sec. 4.1), with an L0 table of one 8-byte
    (sigma 2) or 32-byte (sigma 4) entry per 2^22 lines."""
    from paper_2602_04103_gb300 import capi
    for layout, per in ((3, B2W), (4, B2X)):
        n = 3 * S2 + 5
        idx = build(synth.bits(1, n, 0.5), n, 2, layout)
        info = capi.qr_info(idx)
        nb = n // per + 1
        assert info["bytes_blocks"] == 64 * nb and info["bytes_super"] == 8
        n2 = 1 << 34
        nb = n2 // per + 1
        over = (64 * nb + 8 * ((nb + L0 - 1) // L0)) * 8 / n2 - 1
        assert abs(over * 100 - {3: 6.67, 4: 14.29}[layout]) < 0.01
    idx4 = build(synth.dna_uniform(2, 1000), 1000, 4, 3)
    assert capi.qr_info(idx4)["bytes_super"] == 32
    n4 = 1 << 32
    nb4 = n4 // B4W + 1
    over4 = (64 * nb4 + 32 * ((nb4 + L0 - 1) // L0)) * 8 / (2 * n4) - 1
    assert abs(over4 * 100 - 33.33) < 0.01
    with pytest.raises(capi.QRError):
        build(synth.dna_uniform(2, 1000), 1000, 4, 4)              # BiRank32x2 is sigma 2 only
    # QuadRank24_8 (Sec. 4.1): 33.3% as QuadRank32, its L0 table one 32-byte
    # entry per 2^16 lines
    idx5 = build(synth.dna_uniform(3, 1000), 1000, 4, 5)
    info5 = capi.qr_info(idx5)
    assert info5["bytes_blocks"] == 64 * (1000 // B4W + 1) and info5["bytes_super"] == 32
    assert info5["block_chars"] == B4W and info5["super_blocks"] == L0_24
    over5 = (64 * nb4 + 32 * ((nb4 + L0_24 - 1) // L0_24)) * 8 / (2 * n4) - 1
    assert abs(over5 * 100 - 33.33) < 0.01
    with pytest.raises(capi.QRError):
        build(synth.bits(2, 1000, 0.5), 1000, 2, 5)                # QuadRank24_8 is sigma 4 only
