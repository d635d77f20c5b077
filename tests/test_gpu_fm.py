"""GPU parity of the QuadFm index and counts against the oracle (bit-exact).

The suffix array of T$ is unique, so the GPU's prefix-doubling SA is compared
row by row with the oracle's comparison sort; the BWT, the $ row, C and the
8-mer table follow from their definitions (QuadRank paper, App. D); counts
from the persistent kernel and the per-step baseline are compared with the
oracle's SA-interval counts and brute-force counts.
"""
import itertools

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


def build_fm(codes, keep_sa=True):
    from paper_2602_04103_gb300 import capi
    return capi.qfm_build(dev_u8(codes), codes.size, capi.QFM_KEEP_SA if keep_sa else 0)


def export(idx, n):
    import torch
    from paper_2602_04103_gb300 import capi
    sa = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    bwt = torch.empty(n + 1, dtype=torch.uint8, device="cuda")
    table = torch.empty(2 * 4 ** 8, dtype=torch.int64, device="cuda")
    capi.qfm_export(idx, sa, bwt, table)
    return (sa.cpu().numpy().view(np.uint32).astype(np.uint64), bwt.cpu().numpy(),
            table.cpu().numpy().view(np.uint64).reshape(-1, 2))


def counts(idx, pats, off, stepwise=False):
    import torch
    from paper_2602_04103_gb300 import capi
    m = off.size - 1
    out = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    dp = dev_u8(pats if pats.size else np.zeros(1, np.uint8))
    (capi.qfm_count_stepwise if stepwise else capi.qfm_count)(idx, dp, dev_u64(off), out)
    return host_u64(out)[:m]


def check_index(codes):
    from paper_2602_04103_gb300 import capi
    n = codes.size
    idx = build_fm(codes)
    sa, bwt, table = export(idx, n)
    want_sa = oracle.suffix_array(codes)
    assert np.array_equal(sa, want_sa), np.flatnonzero(sa != want_sa)[:5]
    want_bwt, row = oracle.bwt(codes, want_sa)
    info = capi.qfm_info(idx)
    assert info["dollar_row"] == row
    want_bwt = want_bwt.copy()
    want_bwt[row] = 0          # the $ row is stored as code 0
    assert np.array_equal(bwt, want_bwt)
    assert info["C"] == [1 + int((codes < c).sum()) for c in range(5)]
    # table: SA interval of every 8-mer
    for w in range(0, 4 ** 8, 1 if n < 2000 else 97):
        p = np.array([(w >> (2 * (7 - d))) & 3 for d in range(8)], dtype=np.uint8)
        assert tuple(table[w]) == oracle.sa_interval(codes, want_sa, p), w
    return idx, want_sa


@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 31, 100, 1000])
def test_index_small_random(n):
    rng = np.random.default_rng(n)
    check_index(rng.integers(0, 4, n).astype(np.uint8))


@pytest.mark.parametrize("codes", ["A" * 50, "AC" * 40, "ACGT" * 30, "A" * 30 + "C" + "A" * 30])
def test_index_repetitive(codes):
    check_index(np.array(["ACGT".index(ch) for ch in codes], dtype=np.uint8))


def test_index_planted_repeats():
    t = synth.fm_text(11, 200_000, repeat_cover=0.2, len_min=300, len_max=5000, sub_rate=0.02)
    check_index(t)


def test_counts_tiny_exhaustive():
    # every text of length <= 5 over {A,C}, every pattern of length <= 4 over ACGT
    pats = [np.array(p, dtype=np.uint8) for L in range(0, 5) for p in itertools.product(range(4), repeat=L)]
    off = np.concatenate([[0], np.cumsum([p.size for p in pats])]).astype(np.uint64)
    flat = np.concatenate(pats).astype(np.uint8)
    for L in range(1, 6):
        for t in itertools.product([0, 1], repeat=L):
            t = np.array(t, dtype=np.uint8)
            idx = build_fm(t, keep_sa=False)
            want = oracle.count_brute_batch(t, flat, off)
            assert np.array_equal(counts(idx, flat, off), want), t
            idx.free()


@pytest.mark.parametrize("stepwise", [False, True])
def test_counts_mid_size(stepwise):
    n = 1 << 20
    t = synth.fm_text(21, n)
    idx = build_fm(t)
    sa = oracle.suffix_array(t)
    pats, off = synth.patterns(22, t, 100_000, 1, 150, sub_rate=0.01)
    want = oracle.count_sa(t, sa, pats, off)
    got = counts(idx, pats, off, stepwise=stepwise)
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:5]
    sample = np.arange(0, 100_000, 997)
    sub_off = np.concatenate([[0], np.cumsum(np.diff(off.astype(np.int64))[sample])]).astype(np.uint64)
    sub = np.concatenate([pats[off[k]:off[k + 1]] for k in sample])
    assert np.array_equal(got[sample], oracle.count_brute_batch(t, sub, sub_off))


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_counts_every_l2_policy(policy):
    """The count kernel's L2 policies (plain loads; index evict-last with the
    pattern stream evict-first; index evict-last alone) give the oracle's
    counts, both strands included."""
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 19
    t = synth.fm_text(24, n)
    idx = build_fm(t, keep_sa=False)
    capi.qfm_set_policy(idx, policy)
    pats, off = synth.patterns(25, t, 50_001, 1, 150, sub_rate=0.01)
    want = oracle.count_sa(t, oracle.suffix_array(t), pats, off)
    assert np.array_equal(counts(idx, pats, off), want)
    both = torch.empty(2 * (off.size - 1), dtype=torch.int64, device="cuda")
    capi.qfm_count_ex(idx, dev_u8(pats), dev_u64(off), both, capi.QFM_BOTH_STRANDS)
    assert np.array_equal(host_u64(both)[: off.size - 1], want)
    assert capi.qfm_status(idx) == 0
    with pytest.raises(capi.QRError):
        capi.qfm_set_policy(idx, 3)
    idx.free()


def test_counts_edge_patterns():
    from paper_2602_04103_gb300 import capi
    n = 5000
    t = synth.fm_text(31, n, repeat_cover=0.3, len_min=100, len_max=400)
    idx = build_fm(t)
    sa = oracle.suffix_array(t)
    pl = [np.zeros(0, np.uint8), t[:1], t[:8], t[:9], t[-8:], t[-9:], t.copy(), np.concatenate([t, [0]]),
          t[100:107], t[100:108], t[100:109], np.full(20, 3, np.uint8)]
    off = np.concatenate([[0], np.cumsum([p.size for p in pl])]).astype(np.uint64)
    flat = np.concatenate(pl).astype(np.uint8)
    want = oracle.count_sa(t, sa, flat, off)
    assert want[0] == n + 1 and want[6] == 1 and want[7] == 0
    for stepwise in (False, True):
        assert np.array_equal(counts(idx, flat, off, stepwise), want)
    assert capi.qfm_status(idx) == 0
    # a byte > 3 gives 0 and the bad-symbol status bit
    bad = flat.copy()
    bad[off[3]] = 7
    got = counts(idx, bad, off)
    assert got[3] == 0 and np.array_equal(np.delete(got, 3), np.delete(want, 3))
    assert capi.qfm_status(idx) == capi.QR_EBADSYM
    # empty batch
    assert counts(idx, np.zeros(0, np.uint8), np.zeros(1, np.uint64)).size == 0


def test_build_rejects_bad_text():
    from paper_2602_04103_gb300 import capi
    with pytest.raises(capi.QRError):
        build_fm(np.array([0, 1, 4, 2], dtype=np.uint8))


def test_counts_both_strands():
    import torch
    from paper_2602_04103_gb300 import capi
    n = 1 << 18
    t = synth.fm_text(41, n, repeat_cover=0.2, len_min=300, len_max=2000, sub_rate=0.02)
    idx = build_fm(t, keep_sa=False)
    pats, off = synth.patterns(42, t, 30_000, 1, 150, sub_rate=0.01)
    m = off.size - 1
    out = torch.empty(2 * m, dtype=torch.int64, device="cuda")
    capi.qfm_count_ex(idx, dev_u8(pats), dev_u64(off), out, capi.QFM_BOTH_STRANDS)
    got = host_u64(out)
    assert np.array_equal(got[:m], counts(idx, pats, off))
    sa = oracle.suffix_array(t)
    rc = oracle.revcomp_batch(pats, off)
    assert np.array_equal(got[m:], oracle.count_sa(t, sa, rc, off))
    assert capi.qfm_status(idx) == 0
    with pytest.raises(capi.QRError):
        capi.qfm_count_ex(idx, dev_u8(pats), dev_u64(off), out, 4)


def locate(idx, pats, off):
    """(occ, positions) from qfm_locate: a size query first, then the walk."""
    import torch
    from paper_2602_04103_gb300 import capi
    m = off.size - 1
    occ = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    dp = dev_u8(pats if pats.size else np.zeros(1, np.uint8))
    doff = dev_u64(off)
    total = capi.qfm_locate(idx, dp, doff, occ)
    pos = torch.empty(max(total, 1), dtype=torch.int64, device="cuda")
    assert capi.qfm_locate(idx, dp, doff, occ, pos) == total
    return host_u64(occ), host_u64(pos)[:total]


def plist_batch(t, rng, lengths, per_len, sampled_frac=0.7, extra=()):
    plist = [np.frombuffer(p, np.uint8) for p in extra]
    for L in lengths:
        for _ in range(per_len):
            if rng.random() < sampled_frac and L <= t.size:
                st = int(rng.integers(0, t.size - L + 1))
                plist.append(t[st:st + L])
            else:
                plist.append(rng.integers(0, 4, L).astype(np.uint8))
    off = np.concatenate([[0], np.cumsum([p.size for p in plist])]).astype(np.uint64)
    pats = np.concatenate(plist).astype(np.uint8) if off[-1] else np.zeros(0, np.uint8)
    return pats, off


@pytest.mark.parametrize("sample", [1, 3, 32])
def test_locate_mid_size(sample):
    """Every occurrence's position, in suffix-array row order, equals the
    oracle's SA[lo .. hi) for each pattern (and, sorted, the brute-force scan)."""
    from paper_2602_04103_gb300 import capi
    t = synth.fm_text(71, 20000, repeat_cover=0.3, len_min=100, len_max=2000, sub_rate=0.02)
    idx = capi.qfm_build(dev_u8(t), t.size, 0, sa_sample=sample)
    info = capi.qfm_info(idx)
    assert info["sa_sample"] == sample and info["bytes_locate"] > 0 and not info["has_sa"]
    rng = np.random.default_rng(72)
    pats, off = plist_batch(t, rng, [1, 2, 3, 5, 8, 9, 12, 20, 60], 25, extra=[b""])
    occ, pos = locate(idx, pats, off)
    sa = oracle.suffix_array(t)
    want_occ, want_pos = oracle.locate_sa(t, sa, pats, off)
    assert np.array_equal(occ, want_occ)
    assert np.array_equal(pos, want_pos)
    bocc, bpos = oracle.locate_brute(t, pats, off)
    for k in range(off.size - 1):
        a, b = int(occ[k]), int(occ[k + 1])
        assert np.array_equal(np.sort(pos[a:b]), bpos[a:b]), k
    assert capi.qfm_status(idx) == 0


@pytest.mark.parametrize("sample", [1, 2, 5, 100])
def test_locate_tiny_exhaustive(sample):
    """Every pattern of length 1..4 over small texts, including a sampling
    factor above the text length (only the whole-text suffix is sampled)."""
    from paper_2602_04103_gb300 import capi
    for n, seed in [(1, 1), (9, 2), (40, 3)]:
        t = np.random.default_rng(seed).integers(0, 4, n).astype(np.uint8)
        idx = capi.qfm_build(dev_u8(t), n, 0, sa_sample=sample)
        plist = [np.array(p, np.uint8) for L in range(0, 5) for p in itertools.product(range(4), repeat=L)]
        off = np.concatenate([[0], np.cumsum([p.size for p in plist])]).astype(np.uint64)
        pats = np.concatenate(plist).astype(np.uint8)
        occ, pos = locate(idx, pats, off)
        want_occ, want_pos = oracle.locate_sa(t, oracle.suffix_array(t), pats, off)
        assert np.array_equal(occ, want_occ) and np.array_equal(pos, want_pos), (n, sample)


def test_locate_capacity_and_errors():
    import torch
    from paper_2602_04103_gb300 import capi
    t = synth.fm_text(73, 5000, repeat_cover=0.2, len_min=100, len_max=500, sub_rate=0.02)
    idx = capi.qfm_build(dev_u8(t), t.size, 0, sa_sample=16)
    pats, off = plist_batch(t, np.random.default_rng(74), [1, 4], 10, sampled_frac=1.0)
    bad = np.concatenate([pats, [7, 0, 1]]).astype(np.uint8)      # one pattern with a byte > 3
    boff = np.concatenate([off, [off[-1] + 3]]).astype(np.uint64)
    occ = torch.empty(boff.size, dtype=torch.int64, device="cuda")
    total = capi.qfm_locate(idx, dev_u8(bad), dev_u64(boff), occ)
    assert total == int(oracle.locate_brute(t, pats, off)[0][-1])
    assert host_u64(occ)[-1] == host_u64(occ)[-2] == total         # the malformed pattern has none
    assert capi.qfm_status(idx) == capi.QR_EBADSYM
    small = torch.empty(total - 1, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.QRError) as ei:
        capi.qfm_locate(idx, dev_u8(bad), dev_u64(boff), occ, small)
    assert ei.value.code == capi.QR_ERANGE
    assert host_u64(occ)[-1] == total                              # occ is valid after QR_ERANGE
    plain = capi.qfm_build(dev_u8(t), t.size, 0)                   # built without a sampling factor
    with pytest.raises(capi.QRError):
        capi.qfm_locate(plain, dev_u8(pats), dev_u64(off), occ)
    empty_occ = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    assert capi.qfm_locate(idx, dev_u8(pats), dev_u64(off[:1]), empty_occ) == 0 and host_u64(empty_occ)[0] == 0


def approx_counts(idx, pats, off, k):
    import torch
    from paper_2602_04103_gb300 import capi
    m = off.size - 1
    out = torch.full((max(m, 1),), -1, dtype=torch.int64, device="cuda")
    capi.qfm_count_approx(idx, dev_u8(pats if pats.size else np.zeros(1, np.uint8)), dev_u64(off), k, out)
    return host_u64(out)[:m]


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_count_approx_mid_size(k):
    """Counts with at most k substitutions equal the oracle's window scan;
    k = 0 equals the exact counts."""
    t = synth.fm_text(81, 5000, repeat_cover=0.3, len_min=100, len_max=800, sub_rate=0.02)
    idx = build_fm(t, keep_sa=False)
    rng = np.random.default_rng(82 + k)
    lengths = [1, 2, 3, 6, 9, 14, 25] if k < 3 else [1, 2, 4, 7, 10]
    pats, off = plist_batch(t, rng, lengths, 12, extra=[b""])
    got = approx_counts(idx, pats, off, k)
    assert np.array_equal(got, oracle.count_approx_batch(t, pats, off, k))
    if k == 0:
        assert np.array_equal(got, counts(idx, pats, off))


@pytest.mark.parametrize("k", [1, 2])
def test_count_approx_tiny_exhaustive(k):
    for n, seed in [(1, 5), (12, 6), (50, 7)]:
        t = np.random.default_rng(seed).integers(0, 4, n).astype(np.uint8)
        idx = build_fm(t, keep_sa=False)
        plist = [np.array(p, np.uint8) for L in range(0, 5) for p in itertools.product(range(4), repeat=L)]
        off = np.concatenate([[0], np.cumsum([p.size for p in plist])]).astype(np.uint64)
        pats = np.concatenate(plist).astype(np.uint8)
        assert np.array_equal(approx_counts(idx, pats, off, k), oracle.count_approx_batch(t, pats, off, k)), n


def test_count_approx_repetitive_and_errors():
    from paper_2602_04103_gb300 import capi
    t = np.array([0] * 200 + [1] + [0] * 99, np.uint8)          # A^200 C A^99
    idx = build_fm(t, keep_sa=False)
    plist = [np.zeros(10, np.uint8), np.array([0] * 9 + [1], np.uint8), np.array([2, 3, 1], np.uint8),
             np.array([0, 1, 7], np.uint8)]                     # the last one is malformed
    off = np.concatenate([[0], np.cumsum([p.size for p in plist])]).astype(np.uint64)
    pats = np.concatenate(plist).astype(np.uint8)
    for k in range(4):
        got = approx_counts(idx, pats, off, k)
        want = oracle.count_approx_batch(t, pats[:int(off[3])], off[:4], k)
        assert np.array_equal(got[:3], want) and got[3] == 0, k
    assert capi.qfm_status(idx) == capi.QR_EBADSYM
    import torch
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.QRError):
        capi.qfm_count_approx(idx, dev_u8(pats), dev_u64(off), 4, out)
