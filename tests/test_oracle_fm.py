"""Pins for the FM-side oracle: suffix array, BWT, SA interval counts,
brute-force counts and the LF-step count.

Ties: a hand-worked fixture (GATTACA), Python's own sort of suffix strings,
``re`` overlapping-match counts, closed forms on A^n and (ACGT)^r, and the
extension invariant sum_c count(cP) = count(P) - [T starts with P]
(QuadRank paper, App. D: count-only FM-index with one sentinel).
"""
import re

import numpy as np
import pytest

import oracle
from paper_2602_04103_gb300 import synth

DNA = "ACGT"


def enc(s: str) -> np.ndarray:
    return np.array([DNA.index(ch) for ch in s], dtype=np.uint8)


def dec(a) -> str:
    return "".join(DNA[int(x)] for x in a)


def test_golden_gattaca(golden):
    g = golden("fm_gattaca.txt")
    t = enc(g["text"])
    sa = oracle.suffix_array(t)
    assert sa.tolist() == [int(x) for x in g["sa"].split()]
    bwt, row = oracle.bwt(t, sa)
    assert row == int(g["dollar_row"])
    assert "".join("$" if b == 255 else DNA[b] for b in bwt) == g["bwt"]
    for line in g["pattern"]:
        p, cnt, lo, hi = line.split()
        assert oracle.sa_interval(t, sa, enc(p)) == (int(lo), int(hi))
        assert oracle.count_brute(t, enc(p)) == int(cnt)


@pytest.mark.parametrize("seed,n", [(1, 50), (2, 200), (3, 777)])
def test_sa_matches_python_sort(seed, n):
    rng = np.random.default_rng(seed)
    alpha = 2 if seed == 1 else 4            # a 2-letter text has long repeats
    t = rng.integers(0, alpha, n).astype(np.uint8)
    s = dec(t) + "$"                         # '$' < 'A' < 'C' < 'G' < 'T' in ASCII
    want = sorted(range(n + 1), key=lambda i: s[i:])
    assert oracle.suffix_array(t).tolist() == want


def re_count(text: str, p: str) -> int:
    return len(re.findall("(?=" + p + ")", text))


@pytest.mark.parametrize("seed", [5, 6])
def test_counts_match_regex(seed):
    rng = np.random.default_rng(seed)
    n = 3000
    t = rng.integers(0, 4, n).astype(np.uint8)
    s = dec(t)
    sa = oracle.suffix_array(t)
    for length in [1, 2, 3, 5, 8, 12]:
        for _ in range(20):
            if rng.random() < 0.5:
                st = int(rng.integers(0, n - length + 1))
                p = t[st:st + length]
            else:
                p = rng.integers(0, 4, length).astype(np.uint8)
            want = re_count(s, dec(p))
            assert oracle.count_brute(t, p) == want
            lo, hi = oracle.sa_interval(t, sa, p)
            assert hi - lo == want


def test_closed_forms():
    n = 300
    a = np.zeros(n, dtype=np.uint8)                      # A^n
    sa = oracle.suffix_array(a)
    assert sa.tolist() == list(range(n, -1, -1))         # shorter runs of A sort first
    for k in [0, 1, 7, 8, 150, 300, 301]:
        want = n - k + 1 if k <= n else 0
        assert oracle.count_brute(a, np.zeros(k, np.uint8)) == want
        lo, hi = oracle.sa_interval(a, sa, np.zeros(k, np.uint8))
        assert hi - lo == want
    r = 100
    per = np.tile(np.arange(4, dtype=np.uint8), r)      # (ACGT)^r
    sa = oracle.suffix_array(per)
    for p, want in [("ACGT", r), ("CG", r), ("GTA", r - 1), ("TA", r - 1), ("AA", 0), ("ACGTACGT", r - 1)]:
        lo, hi = oracle.sa_interval(per, sa, enc(p))
        assert hi - lo == want
        assert oracle.count_brute(per, enc(p)) == want


def test_extension_invariant():
    rng = np.random.default_rng(9)
    t = synth.fm_text(77, 4000, repeat_cover=0.3, len_min=50, len_max=200, sub_rate=0.02)
    sa = oracle.suffix_array(t)
    for _ in range(200):
        L = int(rng.integers(0, 10))
        st = int(rng.integers(0, t.size - L))
        p = t[st:st + L]
        cp = oracle.sa_interval(t, sa, p)
        total = 0
        for c in range(4):
            lo, hi = oracle.sa_interval(t, sa, np.concatenate([[c], p]).astype(np.uint8))
            total += hi - lo
        starts = int(L <= t.size and np.array_equal(t[:L], p))
        assert total == (cp[1] - cp[0]) - starts


def test_bwt_definition_and_symbol_counts():
    t = synth.fm_text(3, 2000, repeat_cover=0.2, len_min=100, len_max=300, sub_rate=0.02)
    sa = oracle.suffix_array(t)
    bwt, row = oracle.bwt(t, sa)
    assert sa[row] == 0 and bwt[row] == 255
    # the BWT is a permutation of T$: same symbol multiset
    for c in range(4):
        assert int((bwt == c).sum()) == int((t == c).sum())
    # the row after the last suffix: LF of the $ row maps to row 0 ($ suffix)
    assert sa[0] == t.size


def test_batch_counts_and_steps():
    t = synth.fm_text(5, 5000, repeat_cover=0.2, len_min=300, len_max=1000, sub_rate=0.02)
    sa = oracle.suffix_array(t)
    pats, off = synth.patterns(6, t, 300, 1, 40, sub_rate=0.01)
    a = oracle.count_sa(t, sa, pats, off)
    b = oracle.count_brute_batch(t, pats, off)
    assert np.array_equal(a, b)
    s = dec(t)
    for j in range(0, 300, 37):
        p = dec(pats[off[j]:off[j + 1]])
        assert int(a[j]) == re_count(s, p)
    # LF steps: re-run the loop of a table-then-backward search by brute force
    total, steps = oracle.fm_steps(t, sa, pats, off, k=8)
    assert total == int(steps.sum())
    for j in range(300):
        p = pats[off[j]:off[j + 1]]
        L = p.size
        if L >= 8:
            nonempty = oracle.count_brute(t, p[L - 8:]) > 0
            s_ = 0
            for i in range(L - 9, -1, -1):
                if not nonempty:
                    break
                s_ += 1
                nonempty = oracle.count_brute(t, p[i:]) > 0
        else:
            nonempty, s_ = True, 0
            for i in range(L - 1, -1, -1):
                if not nonempty:
                    break
                s_ += 1
                nonempty = oracle.count_brute(t, p[i:]) > 0
        assert int(steps[j]) == s_, j


def test_revcomp_pins():
    # hand-worked: AACG -> reverse CGAA -> complement (A<->T, C<->G) GCTT
    assert dec(oracle.revcomp(enc("AACG"))) == "CGTT"
    assert dec(oracle.revcomp(enc("GATTACA"))) == "TGTAATC"
    rng = np.random.default_rng(21)
    p = rng.integers(0, 4, 57).astype(np.uint8)
    assert np.array_equal(oracle.revcomp(oracle.revcomp(p)), p)          # an involution
    assert oracle.revcomp(np.zeros(0, np.uint8)).size == 0
    # counting the reverse complement in T = counting the pattern in the other strand of T
    t = synth.fm_text(23, 3000, repeat_cover=0.2, len_min=50, len_max=300, sub_rate=0.02)
    t_rc = oracle.revcomp(t)
    for L in [1, 3, 6, 10]:
        for _ in range(10):
            st = int(rng.integers(0, t.size - L))
            q = t[st:st + L]
            assert oracle.count_brute(t, oracle.revcomp(q)) == oracle.count_brute(t_rc, q)


def test_locate_golden(golden):
    g = golden("fm_gattaca.txt")
    t = enc(g["text"])
    sa = oracle.suffix_array(t)
    for line in g["locate"]:
        f = line.split()
        p = "" if f[0] == "EMPTY" else f[0]
        want = [int(x) for x in f[1:]]
        pats, off = enc(p), np.array([0, len(p)], dtype=np.uint64)
        occ, pos = oracle.locate_sa(t, sa, pats, off)
        assert pos.tolist() == want and occ.tolist() == [0, len(want)]
        occ, pos = oracle.locate_brute(t, pats, off)
        assert pos.tolist() == sorted(want)


def test_locate_matches_regex_and_suffix_order():
    rng = np.random.default_rng(31)
    t = synth.fm_text(41, 3000, repeat_cover=0.3, len_min=50, len_max=300, sub_rate=0.02)
    s = dec(t)
    sa = oracle.suffix_array(t)
    plist = [b""]
    for L in [1, 2, 3, 5, 8, 13, 40]:
        for _ in range(12):
            if rng.random() < 0.7:
                st = int(rng.integers(0, t.size - L))
                plist.append(t[st:st + L].tobytes())
            else:
                plist.append(rng.integers(0, 4, L).astype(np.uint8).tobytes())
    off = np.concatenate([[0], np.cumsum([len(p) for p in plist])]).astype(np.uint64)
    pats = np.frombuffer(b"".join(plist), dtype=np.uint8)
    occ_b, pos_b = oracle.locate_brute(t, pats, off)
    occ_s, pos_s = oracle.locate_sa(t, sa, pats, off)
    assert np.array_equal(occ_b, occ_s)
    assert np.array_equal(np.diff(occ_b), oracle.count_brute_batch(t, pats, off))
    for k, p in enumerate(plist):
        a, b = int(occ_b[k]), int(occ_b[k + 1])
        want = list(range(t.size + 1)) if not p else [mt.start() for mt in re.finditer("(?=" + dec(p) + ")", s)]
        assert pos_b[a:b].tolist() == want
        # suffix-array order: the suffixes at consecutive positions increase ('$' < 'A' in ASCII)
        got = pos_s[a:b].tolist()
        assert sorted(got) == want
        suf = [s[i:] + "$" for i in got]
        assert suf == sorted(suf)


def test_locate_closed_forms():
    n = 200
    a = np.zeros(n, dtype=np.uint8)                       # A^n: A^k starts at 0..n-k
    sa = oracle.suffix_array(a)
    for k in [1, 5, 200, 201]:
        pats, off = np.zeros(k, np.uint8), np.array([0, k], np.uint64)
        want = list(range(n - k + 1)) if k <= n else []
        assert oracle.locate_brute(a, pats, off)[1].tolist() == want
        # rows of A^k are the suffixes A^j$ for j >= k, shortest first: positions n-k, n-k-1, ..., 0
        assert oracle.locate_sa(a, sa, pats, off)[1].tolist() == want[::-1]
    r = 50
    per = np.tile(np.arange(4, dtype=np.uint8), r)       # (ACGT)^r: CG starts at 1, 5, 9, ...
    occ, pos = oracle.locate_brute(per, enc("CG"), np.array([0, 2], np.uint64))
    assert pos.tolist() == list(range(1, 4 * r, 4))


def numpy_hamming_counts(t, p, k):
    """Independent re-statement: sliding windows compared with numpy."""
    L = p.size
    if L == 0:
        return t.size + 1
    if L > t.size:
        return 0
    win = np.lib.stride_tricks.sliding_window_view(t, L)
    return int(((win != p).sum(axis=1) <= k).sum())


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_count_approx_matches_numpy(k):
    rng = np.random.default_rng(50 + k)
    t = synth.fm_text(51, 3000, repeat_cover=0.3, len_min=50, len_max=300, sub_rate=0.02)
    for L in [0, 1, 2, 4, 7, 12, 30]:
        for _ in range(8):
            if L and rng.random() < 0.6:
                st = int(rng.integers(0, t.size - L))
                p = t[st:st + L].copy()
                for j in rng.integers(0, L, int(rng.integers(0, 3))):
                    p[j] = (p[j] + 1 + rng.integers(0, 3)) % 4     # substitute 0..2 chars
            else:
                p = rng.integers(0, 4, L).astype(np.uint8)
            assert oracle.count_approx(t, p, k) == numpy_hamming_counts(t, p, k), (L, k)


def test_count_approx_special_cases():
    rng = np.random.default_rng(60)
    t = rng.integers(0, 4, 2000).astype(np.uint8)
    for L in [1, 5, 11]:
        p = t[100:100 + L]
        assert oracle.count_approx(t, p, 0) == oracle.count_brute(t, p)      # k = 0 is exact count
        assert oracle.count_approx(t, p, L) == t.size - L + 1               # k >= |P|: every window
        cs = [oracle.count_approx(t, p, k) for k in range(4)]
        assert cs == sorted(cs)                                            # monotone in k
    n = 300
    a = np.zeros(n, dtype=np.uint8)                                        # A^n
    p = np.array([0] * 9 + [1], np.uint8)                                  # A^9 C: one substitution from every window
    assert [oracle.count_approx(a, p, k) for k in range(3)] == [0, n - 9, n - 9]
    p = np.array([2, 3, 1], np.uint8)                                      # GTC: three substitutions
    assert [oracle.count_approx(a, p, k) for k in range(4)] == [0, 0, 0, n - 2]
    pats = np.array([0, 0, 1, 2, 0, 3], np.uint8)                          # AA, empty, CG (2 substitutions), AT
    off = np.array([0, 2, 2, 4, 6], np.uint64)
    assert oracle.count_approx_batch(a, pats, off, 1).tolist() == [n - 1, n + 1, 0, n - 1]
