"""The seeded generators: determinism, formats and the stated distributions."""
import numpy as np

from paper_2602_04103_gb300 import synth


def test_splitmix64_reference_values():
    # splitmix64 with state 0 (Vigna's reference implementation): the first
    # output is mix(0x9E3779B97F4A7C15) = 0xE220A8397B1DCDAF.
    assert synth.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    # second output of the same sequential generator: mix(2 * gamma)
    assert synth.splitmix64(0, 1) == 0x6E789E6AA1B965F4


def test_determinism_and_threads():
    a = synth.bits(7, 100_003, 0.3)
    synth.set_threads(1)
    b = synth.bits(7, 100_003, 0.3)
    synth.set_threads(0)
    assert np.array_equal(a, b)
    assert np.array_equal(synth.queries(1, 1000, 5000), synth.queries(1, 1000, 5000))


def test_tail_bits_zero():
    for n in [1, 63, 64, 65, 127]:
        w = synth.bits(3, n, 0.5)
        bits = np.unpackbits(w.view(np.uint8), bitorder="little")
        assert bits[n:].sum() == 0
    for n in [1, 31, 32, 33]:
        w = synth.dna_uniform(3, n)
        assert synth.unpack2(w, (w.size) * 32)[n:].sum() == 0


def test_distributions():
    n = 1 << 20
    for p in [0.5, 0.01]:
        w = synth.bits(9, n, p)
        frac = np.unpackbits(w.view(np.uint8), bitorder="little")[:n].mean()
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / n)
    q = synth.queries(2, 1000, 200_000)
    assert q.max() <= 1000 and q.min() == 0 and (q == 1000).any()
    codes = synth.unpack2(synth.dna_gc_runs(4, n, gc=0.4, run_cover=0.0), n)
    gc = np.isin(codes, [1, 2]).mean()
    assert abs(gc - 0.4) < 0.005
    c = synth.symbols(5, 100_000, 4)
    assert set(np.unique(c).tolist()) == {0, 1, 2, 3}


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    codes = rng.integers(0, 4, 1001).astype(np.uint8)
    assert np.array_equal(synth.unpack2(synth.pack2(codes), 1001), codes)


def test_fm_text_and_patterns():
    t = synth.fm_text(1, 100_000)
    assert t.min() >= 0 and t.max() <= 3
    pats, off = synth.patterns(2, t, 1000, 16, 150, 0.01)
    lens = np.diff(off.astype(np.int64))
    assert lens.min() >= 16 and lens.max() <= 150
    # even patterns are mostly exact substrings (1% substitutions)
    s = t.tobytes()
    hits = sum(s.find(pats[off[k]:off[k + 1]].tobytes()) >= 0 for k in range(0, 200, 2))
    assert hits > 20
