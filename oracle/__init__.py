"""ORACLE -- test infrastructure, not part of the product.

ctypes wrapper over ``oracle.c``: plain CPU definitions of rank, rank_4, the
suffix array / BWT of T$, pattern occurrence counts (exact and with up to k
substitutions) and positions (QuadRank paper, Sec. 1 rank definition and
approximate matching, Sec. 4 rank_4, App. D count-only FM-index, Sec. 6
locate).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
in ``paper_2602_04103_gb300``; both only consume the seeded inputs of
``paper_2602_04103_gb300.synth``.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, library routines or brute force.
"""
from __future__ import annotations

import ctypes as C
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
SO = HERE / "_lib" / "liboracle.so"

OR_OK, OR_EINVAL, OR_ENOMEM, OR_ERANGE = 0, 1, 2, 4
U64_MAX = np.uint64(0xFFFFFFFFFFFFFFFF)

_lib = None
u64 = C.c_uint64
_P = C.c_void_p


def build(force: bool = False) -> Path:
    """Compile liboracle.so with gcc (portable C, no ISA-specific flags)."""
    SO.parent.mkdir(exist_ok=True)
    if force or not SO.exists() or SO.stat().st_mtime < SRC.stat().st_mtime:
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(SRC), "-o", str(SO)],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    return SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(str(SO))
        lib.or_char.restype = u64
        lib.or_char.argtypes = [_P, C.c_int, u64]
        lib.or_rank_naive.argtypes = [_P, u64, C.c_int, u64, C.c_int, _P]
        lib.or_rank_sweep.argtypes = [_P, u64, C.c_int, _P, u64, C.c_int, C.c_int, _P, _P]
        lib.or_rank_sweep_mt.argtypes = [_P, u64, C.c_int, _P, u64, C.c_int, C.c_int, _P, _P, C.c_int]
        lib.or_suffix_array.argtypes = [_P, u64, _P]
        lib.or_bwt.argtypes = [_P, u64, _P, _P, _P]
        lib.or_sa_interval.argtypes = [_P, u64, _P, _P, u64, _P, _P]
        lib.or_count_brute.restype = u64
        lib.or_count_brute.argtypes = [_P, u64, _P, u64]
        lib.or_count_sa.argtypes = [_P, u64, _P, _P, _P, u64, _P]
        lib.or_count_brute_batch.argtypes = [_P, u64, _P, _P, u64, _P]
        lib.or_revcomp.argtypes = [_P, u64, _P]
        lib.or_locate_brute.argtypes = [_P, u64, _P, _P, u64, _P, _P]
        lib.or_count_approx.restype = u64
        lib.or_count_approx.argtypes = [_P, u64, _P, u64, C.c_uint32]
        lib.or_count_approx_batch.argtypes = [_P, u64, _P, _P, u64, C.c_uint32, _P]
        lib.or_locate_sa.argtypes = [_P, u64, _P, _P, _P, u64, _P, _P]
        lib.or_rank_chain.argtypes = [_P, u64, C.c_int, _P, u64, u64, C.c_int, _P]
        lib.or_fm_steps.restype = u64
        lib.or_fm_steps.argtypes = [_P, u64, _P, _P, _P, u64, u64, _P]
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def char(text: np.ndarray, sigma: int, i: int) -> int:
    return int(_load().or_char(_p(_u64(text)), sigma, i))


def rank_naive(text: np.ndarray, n: int, sigma: int, q: int, c: int) -> int:
    text = _u64(text)
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().or_rank_naive(_p(text), n, sigma, q, c, _p(out))
    if rc != OR_OK:
        raise ValueError(f"or_rank_naive rc={rc}")
    return int(out[0])


def _sweep(text, n, sigma, q, mode, c, c_arr, out, threads):
    """or_rank_sweep, or its threaded form when threads > 1."""
    lib = _load()
    cp = _p(c_arr) if c_arr is not None else None
    if threads > 1:
        return lib.or_rank_sweep_mt(_p(text), n, sigma, _p(q), q.size, mode, c, cp, _p(out), threads)
    return lib.or_rank_sweep(_p(text), n, sigma, _p(q), q.size, mode, c, cp, _p(out))


def rank(text: np.ndarray, n: int, sigma: int, q: np.ndarray, c: int, threads: int = 1) -> tuple[np.ndarray, int]:
    """rank(q[k], c) for every k by one sweep (on `threads` threads); returns (out, rc)."""
    text, q = _u64(text), _u64(q)
    out = np.empty(q.size, dtype=np.uint64)
    return out, _sweep(text, n, sigma, q, 0, c, None, out, threads)


def rank_c(text: np.ndarray, n: int, sigma: int, q: np.ndarray, c: np.ndarray,
           threads: int = 1) -> tuple[np.ndarray, int]:
    text, q, c = _u64(text), _u64(q), _u8(c)
    out = np.empty(q.size, dtype=np.uint64)
    return out, _sweep(text, n, sigma, q, 1, 0, c, out, threads)


def rank4(text: np.ndarray, n: int, q: np.ndarray, threads: int = 1) -> tuple[np.ndarray, int]:
    text, q = _u64(text), _u64(q)
    out = np.empty((q.size, 4), dtype=np.uint64)
    return out, _sweep(text, n, 4, q, 2, 0, None, out, threads)


def prefix_rank(text: np.ndarray, n: int, sigma: int, q: np.ndarray, c: int,
                threads: int = 1) -> tuple[np.ndarray, int]:
    """#{i < q[k] : t_i <= c} for every k by one sweep; returns (out, rc)."""
    text, q = _u64(text), _u64(q)
    out = np.empty(q.size, dtype=np.uint64)
    return out, _sweep(text, n, sigma, q, 3, c, None, out, threads)


def rank_chain(text: np.ndarray, n: int, sigma: int, q0: np.ndarray, steps: int, c: int) -> tuple[np.ndarray, int]:
    """Dependent query chains: (out[chains, 2] = last position, last rank; rc)."""
    text, q0 = _u64(text), _u64(q0)
    out = np.empty((q0.size, 2), dtype=np.uint64)
    rc = _load().or_rank_chain(_p(text), n, sigma, _p(q0), q0.size, steps, c, _p(out))
    return out, rc


def suffix_array(codes: np.ndarray) -> np.ndarray:
    codes = _u8(codes)
    sa = np.empty(codes.size + 1, dtype=np.uint64)
    _load().or_suffix_array(_p(codes), codes.size, _p(sa))
    return sa


def bwt(codes: np.ndarray, sa: np.ndarray) -> tuple[np.ndarray, int]:
    """(bwt bytes with 255 at the $ row, $ row)."""
    codes, sa = _u8(codes), _u64(sa)
    out = np.empty(codes.size + 1, dtype=np.uint8)
    row = np.zeros(1, dtype=np.uint64)
    _load().or_bwt(_p(codes), codes.size, _p(sa), _p(out), _p(row))
    return out, int(row[0])


def sa_interval(codes: np.ndarray, sa: np.ndarray, p: np.ndarray) -> tuple[int, int]:
    codes, sa, p = _u8(codes), _u64(sa), _u8(p)
    lo = np.zeros(1, dtype=np.uint64)
    hi = np.zeros(1, dtype=np.uint64)
    _load().or_sa_interval(_p(codes), codes.size, _p(sa), _p(p) if p.size else None, p.size, _p(lo), _p(hi))
    return int(lo[0]), int(hi[0])


def count_brute(codes: np.ndarray, p: np.ndarray) -> int:
    codes, p = _u8(codes), _u8(p)
    return int(_load().or_count_brute(_p(codes), codes.size, _p(p) if p.size else None, p.size))


def count_brute_batch(codes: np.ndarray, pats: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    codes, pats, offsets = _u8(codes), _u8(pats), _u64(offsets)
    m = offsets.size - 1
    out = np.empty(m, dtype=np.uint64)
    _load().or_count_brute_batch(_p(codes), codes.size, _p(pats) if pats.size else None, _p(offsets), m, _p(out))
    return out


def count_sa(codes: np.ndarray, sa: np.ndarray, pats: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    codes, sa, pats, offsets = _u8(codes), _u64(sa), _u8(pats), _u64(offsets)
    m = offsets.size - 1
    out = np.empty(m, dtype=np.uint64)
    _load().or_count_sa(_p(codes), codes.size, _p(sa), _p(pats) if pats.size else None, _p(offsets), m, _p(out))
    return out


def count_approx(codes: np.ndarray, p: np.ndarray, k: int) -> int:
    """Positions where P matches with at most k substitutions."""
    codes, p = _u8(codes), _u8(p)
    return int(_load().or_count_approx(_p(codes), codes.size, _p(p) if p.size else None, p.size, k))


def count_approx_batch(codes: np.ndarray, pats: np.ndarray, offsets: np.ndarray, k: int) -> np.ndarray:
    codes, pats, offsets = _u8(codes), _u8(pats), _u64(offsets)
    m = offsets.size - 1
    out = np.empty(m, dtype=np.uint64)
    _load().or_count_approx_batch(_p(codes), codes.size, _p(pats) if pats.size else None, _p(offsets), m, k, _p(out))
    return out


def locate_brute(codes: np.ndarray, pats: np.ndarray, offsets: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(occ[m+1], positions): every start position of each pattern, increasing."""
    codes, pats, offsets = _u8(codes), _u8(pats), _u64(offsets)
    m = offsets.size - 1
    occ = np.empty(m + 1, dtype=np.uint64)
    lib = _load()
    pp = _p(pats) if pats.size else None
    lib.or_locate_brute(_p(codes), codes.size, pp, _p(offsets), m, _p(occ), None)
    pos = np.empty(max(int(occ[m]), 1), dtype=np.uint64)
    lib.or_locate_brute(_p(codes), codes.size, pp, _p(offsets), m, _p(occ), _p(pos))
    return occ, pos[: int(occ[m])]


def locate_sa(codes: np.ndarray, sa: np.ndarray, pats: np.ndarray, offsets: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(occ[m+1], positions): each pattern's positions in suffix-array row order."""
    codes, sa, pats, offsets = _u8(codes), _u64(sa), _u8(pats), _u64(offsets)
    m = offsets.size - 1
    occ = np.empty(m + 1, dtype=np.uint64)
    lib = _load()
    pp = _p(pats) if pats.size else None
    lib.or_locate_sa(_p(codes), codes.size, _p(sa), pp, _p(offsets), m, _p(occ), None)
    pos = np.empty(max(int(occ[m]), 1), dtype=np.uint64)
    lib.or_locate_sa(_p(codes), codes.size, _p(sa), pp, _p(offsets), m, _p(occ), _p(pos))
    return occ, pos[: int(occ[m])]


def fm_steps(codes: np.ndarray, sa: np.ndarray, pats: np.ndarray, offsets: np.ndarray,
             k: int = 8) -> tuple[int, np.ndarray]:
    codes, sa, pats, offsets = _u8(codes), _u64(sa), _u8(pats), _u64(offsets)
    m = offsets.size - 1
    steps = np.empty(m, dtype=np.uint64)
    total = _load().or_fm_steps(_p(codes), codes.size, _p(sa), _p(pats) if pats.size else None,
                                _p(offsets), m, k, _p(steps))
    return int(total), steps


def revcomp(p: np.ndarray) -> np.ndarray:
    p = _u8(p)
    out = np.empty(p.size, dtype=np.uint8)
    if p.size:
        _load().or_revcomp(_p(p), p.size, _p(out))
    return out


def revcomp_batch(pats: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Reverse complement of every pattern of a batch (same offsets)."""
    pats, offsets = _u8(pats), _u64(offsets)
    out = np.empty_like(pats)
    for k in range(offsets.size - 1):
        a, b = int(offsets[k]), int(offsets[k + 1])
        out[a:b] = revcomp(pats[a:b])
    return out
