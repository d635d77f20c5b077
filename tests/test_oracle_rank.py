"""Pins for the rank oracle (rank, rank_c, rank4, rank_naive).

Each check ties the oracle to something other than itself: hand-worked
fixtures, closed forms of structured texts, numpy prefix sums of the
unpacked text, and the invariants that define rank (QuadRank paper, Sec. 1:
rank(q, c) = #{i < q : t_i = c}; Sec. 4: rank_4 returns all four symbols).
"""
import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth

DNA = {"A": 0, "C": 1, "G": 2, "T": 3}


def test_golden_bits(golden):
    g = golden("rank_bits_16.txt")
    bits = np.array([int(ch) for ch in g["text"]], dtype=np.uint8)
    words = synth.pack_bits(bits)
    assert int(words[0]) == int(g["word"], 16)
    want = [int(x) for x in g["rank1"].split()]
    n = bits.size
    q = np.arange(n + 1, dtype=np.uint64)
    got, rc = oracle.rank(words, n, 2, q, 1)
    assert rc == 0 and got.tolist() == want
    got0, _ = oracle.rank(words, n, 2, q, 0)
    assert got0.tolist() == [k - r for k, r in zip(range(n + 1), want)]
    for k in range(n + 1):
        assert oracle.rank_naive(words, n, 2, k, 1) == want[k]


def test_golden_dna(golden):
    g = golden("rank_dna_gattaca.txt")
    codes = np.array([DNA[ch] for ch in g["text"]], dtype=np.uint8)
    words = synth.pack2(codes)
    assert int(words[0]) == int(g["word"], 16)
    n = codes.size
    q = np.arange(n + 1, dtype=np.uint64)
    r4, rc = oracle.rank4(words, n, q)
    assert rc == 0
    for sym, c in DNA.items():
        want = [int(x) for x in g["rank" + sym].split()]
        got, rc = oracle.rank(words, n, 4, q, c)
        assert rc == 0 and got.tolist() == want
        assert r4[:, c].tolist() == want
        assert [oracle.rank_naive(words, n, 4, k, c) for k in range(n + 1)] == want


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 4099])
def test_closed_forms_bits(n):
    q = np.arange(n + 1, dtype=np.uint64)
    ones = synth.pack_bits(np.ones(n, dtype=np.uint8))
    assert oracle.rank(ones, n, 2, q, 1)[0].tolist() == list(range(n + 1))
    assert oracle.rank(ones, n, 2, q, 0)[0].tolist() == [0] * (n + 1)
    sparse = np.array([0, n // 3, n], dtype=np.uint64)
    assert oracle.rank(ones, n, 2, sparse, 0)[0].tolist() == [0, 0, 0]
    assert oracle.rank(ones, n, 2, sparse, 1)[0].tolist() == sparse.tolist()
    zeros = synth.pack_bits(np.zeros(n, dtype=np.uint8))
    assert oracle.rank(zeros, n, 2, q, 1)[0].tolist() == [0] * (n + 1)
    assert oracle.rank(zeros, n, 2, sparse, 0)[0].tolist() == sparse.tolist()
    alt = synth.pack_bits((np.arange(n) % 2 == 0).astype(np.uint8))   # 1 0 1 0 ...
    assert oracle.rank(alt, n, 2, q, 1)[0].tolist() == [(k + 1) // 2 for k in range(n + 1)]
    p3 = synth.pack_bits((np.arange(n) % 3 != 2).astype(np.uint8))    # 1 1 0 1 1 0 ...
    assert oracle.rank(p3, n, 2, q, 1)[0].tolist() == [2 * (k // 3) + min(k % 3, 2) for k in range(n + 1)]


@pytest.mark.parametrize("n", [1, 31, 32, 33, 997, 4100])
def test_closed_forms_dna(n):
    q = np.arange(n + 1, dtype=np.uint64)
    period = synth.pack2((np.arange(n) % 4).astype(np.uint8))        # ACGTACGT...
    r4, rc = oracle.rank4(period, n, q)
    assert rc == 0
    for c in range(4):
        assert r4[:, c].tolist() == [(k + 3 - c) // 4 for k in range(n + 1)]
    # runs: A^a C^b G^c T^rest
    a, b, cc = n // 4, n // 3, n // 5
    codes = np.concatenate([np.full(a, 0), np.full(b, 1), np.full(cc, 2), np.full(n - a - b - cc, 3)]).astype(np.uint8)
    w = synth.pack2(codes)
    edges = [0, a, a + b, a + b + cc, n]
    r4, _ = oracle.rank4(w, n, q)
    for c in range(4):
        want = [min(max(k - edges[c], 0), edges[c + 1] - edges[c]) for k in range(n + 1)]
        assert r4[:, c].tolist() == want


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_numpy_prefix_sums_bits(seed):
    n = 9000 + seed * 17
    words = synth.bits(seed, n, p=[0.5, 0.1, 0.9][seed - 1])
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:n].astype(np.uint64)
    pref = np.concatenate([[0], np.cumsum(bits)]).astype(np.uint64)
    q = np.arange(n + 1, dtype=np.uint64)
    got, rc = oracle.rank(words, n, 2, q, 1)
    assert rc == 0 and np.array_equal(got, pref)
    got0, _ = oracle.rank(words, n, 2, q, 0)
    assert np.array_equal(got0, q - pref)
    # sparse queries: the sweep then crosses whole 64-bit words between answers
    qs = synth.queries(seed + 100, n, 60)
    for c, want in [(1, pref[qs]), (0, qs - pref[qs])]:
        got, rc = oracle.rank(words, n, 2, qs, c)
        assert rc == 0 and np.array_equal(got, want)


@pytest.mark.parametrize("seed", [4, 5])
def test_numpy_prefix_sums_dna(seed):
    n = 7001 + seed
    rng = np.random.default_rng(seed)
    codes = rng.integers(0, 4, n).astype(np.uint8)
    words = synth.pack2(codes)
    q = np.arange(n + 1, dtype=np.uint64)
    r4, rc = oracle.rank4(words, n, q)
    assert rc == 0
    for c in range(4):
        pref = np.concatenate([[0], np.cumsum(codes == c)]).astype(np.uint64)
        assert np.array_equal(r4[:, c], pref)
        got, _ = oracle.rank(words, n, 4, q, c)
        assert np.array_equal(got, pref)


@pytest.mark.parametrize("sigma", [2, 4])
def test_invariants_random_text(sigma):
    n = 20000
    words = synth.bits(11, n, 0.5) if sigma == 2 else synth.dna_uniform(12, n)
    q = np.arange(n + 1, dtype=np.uint64)
    ranks = np.stack([oracle.rank(words, n, sigma, q, c)[0] for c in range(sigma)], axis=1).astype(np.int64)
    assert (ranks[0] == 0).all()                                   # rank(0, c) = 0
    assert (ranks.sum(axis=1) == np.arange(n + 1)).all()            # sum_c rank(q, c) = q
    diff = np.diff(ranks, axis=0)
    assert ((diff == 0) | (diff == 1)).all()                        # monotone, unit steps
    t = np.array([oracle.char(words, sigma, i) for i in range(0, n, 97)])
    # rank(q+1, c) - rank(q, c) = [t_q = c]
    for j, i in enumerate(range(0, n, 97)):
        assert diff[i].tolist() == [int(t[j] == c) for c in range(sigma)]


def test_per_query_symbols_and_range():
    n = 5000
    words = synth.dna_uniform(21, n)
    q = synth.queries(22, n, 3000)
    c = synth.symbols(23, 3000, 4)
    got, rc = oracle.rank_c(words, n, 4, q, c)
    assert rc == 0
    r4, _ = oracle.rank4(words, n, q)
    assert np.array_equal(got, r4[np.arange(q.size), c])
    # out of range: q > n gives UINT64_MAX and OR_ERANGE
    bad = np.array([0, n, n + 1, 2 ** 63], dtype=np.uint64)
    got, rc = oracle.rank(words, n, 4, bad, 2)
    assert rc == oracle.OR_ERANGE
    assert got[2] == oracle.U64_MAX and got[3] == oracle.U64_MAX
    assert got[0] == 0


def test_sweep_matches_naive_unsorted_duplicates():
    n = 3001
    words = synth.bits(31, n, 0.3)
    q = np.array([n, 0, 17, 17, 64, 63, 65, n, 1, 3000, 128, 127], dtype=np.uint64)
    got, rc = oracle.rank(words, n, 2, q, 1)
    assert rc == 0
    assert got.tolist() == [oracle.rank_naive(words, n, 2, int(x), 1) for x in q]


def test_prefix_rank_pins(golden):
    # GATTACA by hand: chars <= C (A or C) before q = rankA + rankC from the fixture
    g = golden("rank_dna_gattaca.txt")
    codes = np.array([DNA[ch] for ch in g["text"]], dtype=np.uint8)
    words = synth.pack2(codes)
    q = np.arange(8, dtype=np.uint64)
    want = [int(a) + int(b) for a, b in zip(g["rankA"].split(), g["rankC"].split())]
    got, rc = oracle.prefix_rank(words, 7, 4, q, 1)
    assert rc == 0 and got.tolist() == want
    # numpy: cumulative count of codes <= c; c = 3 gives q
    rng = np.random.default_rng(77)
    codes = rng.integers(0, 4, 5003).astype(np.uint8)
    words = synth.pack2(codes)
    q = np.arange(5004, dtype=np.uint64)
    for c in range(4):
        pref = np.concatenate([[0], np.cumsum(codes <= c)]).astype(np.uint64)
        assert np.array_equal(oracle.prefix_rank(words, 5003, 4, q, c)[0], pref)
    assert np.array_equal(oracle.prefix_rank(words, 5003, 4, q, 3)[0], q)


def test_rank_chain_pins():
    # every step of a chain: rank by the definition loop, the next position by the chain rule
    n = 3001
    words = synth.bits(81, n, 0.4)
    q0 = np.array([0, 5, n, 1234], dtype=np.uint64)
    steps = 7
    got, rc = oracle.rank_chain(words, n, 2, q0, steps, 1)
    assert rc == 0
    for k, q in enumerate(q0.tolist()):
        r = 0
        for t in range(steps):
            r = oracle.rank_naive(words, n, 2, q, 1)
            if t + 1 < steps:
                q = ((((q + r) * 0x9E3779B97F4A7C15) % 2 ** 64) * (n + 1)) >> 64
        assert got[k].tolist() == [q, r]
    bad, rc = oracle.rank_chain(words, n, 2, np.array([n + 1], dtype=np.uint64), 3, 1)
    assert rc == oracle.OR_ERANGE and bad[0, 0] == oracle.U64_MAX


@pytest.mark.parametrize("threads", [2, 3, 8, 33])
def test_threaded_sweep_numpy_prefix_sums(threads):
    # the threaded sweep (text cut into chunks answered side by side) against
    # numpy prefix sums of the unpacked text, every q and all modes
    n = 9001
    words = synth.bits(3, n, 0.3)
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:n].astype(np.uint64)
    pref = np.concatenate([[0], np.cumsum(bits)]).astype(np.uint64)
    q = synth.queries(5, n, 20000)
    q[:3] = [0, n, n]
    got, rc = oracle.rank(words, n, 2, q, 1, threads=threads)
    assert rc == 0 and np.array_equal(got, pref[q])
    got0, rc = oracle.rank(words, n, 2, q, 0, threads=threads)
    assert rc == 0 and np.array_equal(got0, q - pref[q])
    rng = np.random.default_rng(threads)
    codes = rng.integers(0, 4, 7003).astype(np.uint8)
    w4 = synth.pack2(codes)
    q4 = np.arange(7004, dtype=np.uint64)[::-1].copy()        # every q, descending
    prefs = [np.concatenate([[0], np.cumsum(codes == c)]).astype(np.uint64) for c in range(4)]
    r4, rc = oracle.rank4(w4, 7003, q4, threads=threads)
    assert rc == 0
    for c in range(4):
        assert np.array_equal(r4[:, c], prefs[c][q4])
        assert np.array_equal(oracle.rank(w4, 7003, 4, q4, c, threads=threads)[0], prefs[c][q4])
        le = sum(prefs[k] for k in range(c + 1))
        assert np.array_equal(oracle.prefix_rank(w4, 7003, 4, q4, c, threads=threads)[0], le[q4])
    cs = synth.symbols(6, q4.size, 4)
    got, rc = oracle.rank_c(w4, 7003, 4, q4, cs, threads=threads)
    assert rc == 0 and np.array_equal(got, r4[np.arange(q4.size), cs])


@pytest.mark.parametrize("threads", [2, 5, 64])
def test_threaded_sweep_equals_single_edges(threads):
    # tiny texts (fewer positions than threads), closed forms, q = n, errors
    for n in (1, 7, 64, 65, 130):
        ones = synth.pack_bits(np.ones(n, dtype=np.uint8))
        q = np.arange(n + 1, dtype=np.uint64)
        got, rc = oracle.rank(ones, n, 2, q, 1, threads=threads)
        assert rc == 0 and got.tolist() == list(range(n + 1))
    n = 5000
    words = synth.dna_uniform(21, n)
    bad = np.array([0, n, n + 1, 2 ** 63, 17], dtype=np.uint64)
    got, rc = oracle.rank(words, n, 4, bad, 2, threads=threads)
    want, rc1 = oracle.rank(words, n, 4, bad, 2)
    assert rc == rc1 == oracle.OR_ERANGE and np.array_equal(got, want)
    syms = np.array([0, 1, 4, 3, 2], dtype=np.uint8)          # one symbol out of range
    q = np.array([5, 6, 7, 8, 9], dtype=np.uint64)
    got, rc = oracle.rank_c(words, n, 4, q, syms, threads=threads)
    want, rc1 = oracle.rank_c(words, n, 4, q, syms)
    assert rc == rc1 == oracle.OR_EINVAL and np.array_equal(got, want)
    r4, rc = oracle.rank4(words, n, bad, threads=threads)
    w4, rc1 = oracle.rank4(words, n, bad)
    assert rc == rc1 and np.array_equal(r4, w4)
