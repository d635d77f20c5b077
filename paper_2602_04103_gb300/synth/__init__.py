"""Seeded synthetic inputs (numpy arrays) drawn by ``libqrsynth.so``.

Shared by the oracle side (tests, CPU baseline) and the CUDA side (tests,
benchmark): the generators hold no rank or search arithmetic, only the draws
and the packing formats of the C-ABI.

Seeds: every workload has a base seed ``0x5EED0000 + workload_id``; its
sub-streams are ``substream(base, k)`` with k = 1 text, 2 queries, 3 symbols,
(pattern sets use ``substream(base, 4/5)`` inside the C code).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_SO = Path(__file__).resolve().parent / "libqrsynth.so"
_lib = None

u64 = C.c_uint64
_P = C.c_void_p


def _load():
    global _lib
    if _lib is None:
        if not _SO.exists():
            from .. import _build
            _build.build_synth()
        lib = C.CDLL(str(_SO))
        lib.qs_splitmix64.restype = u64
        lib.qs_splitmix64.argtypes = [u64, u64]
        lib.qs_substream.restype = u64
        lib.qs_substream.argtypes = [u64, u64]
        lib.qs_bits.argtypes = [u64, u64, C.c_double, _P]
        lib.qs_dna_uniform.argtypes = [u64, u64, _P]
        lib.qs_dna_gc_runs.argtypes = [u64, u64, C.c_double, C.c_double, u64, u64, _P]
        lib.qs_queries.argtypes = [u64, u64, u64, _P]
        lib.qs_symbols.argtypes = [u64, u64, C.c_int, _P]
        lib.qs_pack2.argtypes = [_P, u64, _P]
        lib.qs_unpack2.argtypes = [_P, u64, _P]
        lib.qs_fm_text.argtypes = [u64, u64, C.c_double, u64, u64, C.c_double, _P]
        lib.qs_pattern_offsets.restype = u64
        lib.qs_pattern_offsets.argtypes = [u64, u64, u64, u64, _P]
        lib.qs_patterns.argtypes = [u64, _P, u64, u64, _P, C.c_double, _P]
        lib.qs_set_threads.argtypes = [C.c_int]
        lib.qs_threads.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def base_seed(workload_id: int) -> int:
    return 0x5EED0000 + int(workload_id)


def splitmix64(seed: int, i: int) -> int:
    return int(_load().qs_splitmix64(seed, i))


def substream(seed: int, k: int) -> int:
    return int(_load().qs_substream(seed, k))


def bits(seed: int, n: int, p: float = 0.5) -> np.ndarray:
    """i.i.d. bits with P(1)=p, packed LSB-first in ceil(n/64) uint64 words (+1 zero pad word)."""
    w = np.zeros((n + 63) // 64 + 1, dtype=np.uint64)
    _load().qs_bits(seed, n, p, _ptr(w))
    return w


def dna_uniform(seed: int, n: int) -> np.ndarray:
    """i.i.d. uniform DNA, 2-bit packed in ceil(n/32) uint64 words (+1 zero pad word)."""
    w = np.zeros((n + 31) // 32 + 1, dtype=np.uint64)
    _load().qs_dna_uniform(seed, n, _ptr(w))
    return w


def dna_gc_runs(seed: int, n: int, gc: float = 0.4, run_cover: float = 0.05,
                run_min: int = 10, run_max: int = 1000) -> np.ndarray:
    w = np.zeros((n + 31) // 32 + 1, dtype=np.uint64)
    _load().qs_dna_gc_runs(seed, n, gc, run_cover, run_min, run_max, _ptr(w))
    return w


def queries(seed: int, n: int, m: int) -> np.ndarray:
    """m positions uniform in [0, n]."""
    q = np.empty(m, dtype=np.uint64)
    _load().qs_queries(seed, n, m, _ptr(q))
    return q


def symbols(seed: int, m: int, sigma: int) -> np.ndarray:
    c = np.empty(m, dtype=np.uint8)
    if _load().qs_symbols(seed, m, sigma, _ptr(c)) != 0:
        raise ValueError("sigma must be 2 or 4")
    return c


def pack2(codes: np.ndarray) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    n = codes.size
    w = np.zeros((n + 31) // 32 + 1, dtype=np.uint64)
    _load().qs_pack2(_ptr(codes), n, _ptr(w))
    return w


def unpack2(words: np.ndarray, n: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint64)
    c = np.empty(n, dtype=np.uint8)
    _load().qs_unpack2(_ptr(words), n, _ptr(c))
    return c


def pack_bits(bits01: np.ndarray) -> np.ndarray:
    """Pack a 0/1 array LSB-first into uint64 words (+1 zero pad word)."""
    b = np.ascontiguousarray(bits01, dtype=np.uint8)
    n = b.size
    w = np.zeros((n + 63) // 64 + 1, dtype=np.uint64)
    by = np.packbits(b, bitorder="little")
    w.view(np.uint8)[: by.size] = by
    return w


def fm_text(seed: int, n: int, repeat_cover: float = 0.2, len_min: int = 300, len_max: int = 5000,
            sub_rate: float = 0.02) -> np.ndarray:
    """Uniform DNA codes (uint8) with planted repeats."""
    c = np.empty(n, dtype=np.uint8)
    if _load().qs_fm_text(seed, n, repeat_cover, len_min, len_max, sub_rate, _ptr(c)) != 0:
        raise MemoryError("qs_fm_text")
    return c


def patterns(seed: int, text: np.ndarray, m: int, len_min: int, len_max: int,
             sub_rate: float = 0.01) -> tuple[np.ndarray, np.ndarray]:
    """(codes uint8, offsets uint64[m+1]); even patterns sampled from text with substitutions."""
    text = np.ascontiguousarray(text, dtype=np.uint8)
    off = np.empty(m + 1, dtype=np.uint64)
    total = int(_load().qs_pattern_offsets(seed, m, len_min, len_max, _ptr(off)))
    pat = np.empty(max(total, 1), dtype=np.uint8)
    _load().qs_patterns(seed, _ptr(text), text.size, m, _ptr(off), sub_rate, _ptr(pat))
    return pat[:total], off


def set_threads(t: int) -> None:
    _load().qs_set_threads(int(t))


def threads() -> int:
    return int(_load().qs_threads())
