"""Write the expected values of the full-size QuadFm parity tests, computed by
the oracle only (count-only FM-index, QuadRank paper App. D):

fm_full_2p26_1e7.json -- the count workload: 2^26-char text with 20% planted
  repeats, 10^7 patterns of length 16..150.
  * sha256 of the suffix array of T$ (textbook comparison sort, as uint32),
  * sha256 of all 10^7 counts (suffix-array interval sizes, as uint64),
  * sha256 of the counts of the reverse complements of 10^5 sampled patterns
    (both-strand counting, App. D counts each read in both directions),
  * plain sums and a few leading values, for a readable diff.
fm_serving_2p28.json -- the serving workload: 2^28-char text, the first
  256 requests of the trace; brute-force counts (direct comparison at every
  text position) of 2000 sampled patterns of those requests.

Hashes are of little-endian arrays.  The oracle calls run on all host cores
(each thread calls the single-threaded C oracle on its own slice of the
patterns; ctypes releases the interpreter lock during a call).

Run:  python tests/golden/make_fm_full.py   (about 5-10 minutes on 8 cores)
"""
import hashlib
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2602_04103_gb300 import workloads  # noqa: E402

HERE = Path(__file__).resolve().parent
SERVE_REQUESTS = 256
SERVE_SAMPLE = 2000
BOTH_SAMPLE = 100_000


def sha(a: np.ndarray, dtype: str) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def sub_batch(pats: np.ndarray, off: np.ndarray, ids: np.ndarray):
    """The patterns `ids` of a batch as a batch of their own."""
    lens = (off[ids + 1] - off[ids]).astype(np.int64)
    sub = np.concatenate([pats[int(off[k]):int(off[k + 1])] for k in ids]) if ids.size else np.zeros(0, np.uint8)
    sub_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    return sub, sub_off


def threaded(fn, m: int, threads: int) -> np.ndarray:
    """fn(a, b) -> counts of patterns a..b, over `threads` slices."""
    cuts = np.linspace(0, m, threads * 4 + 1).astype(np.int64)
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda k: fn(int(cuts[k]), int(cuts[k + 1])), range(cuts.size - 1)))
    return np.concatenate(parts) if parts else np.zeros(0, np.uint64)


def count_workload(threads: int) -> dict:
    t0 = time.time()
    text, pats, off = workloads.fm_inputs()
    m = off.size - 1
    sa = oracle.suffix_array(text)
    t_sa = time.time() - t0

    def counts(a, b):
        return oracle.count_sa(text, sa, pats[int(off[a]):int(off[b])], (off[a:b + 1] - off[a]).astype(np.uint64))

    cnt = threaded(counts, m, threads)
    both_ids = workloads.sample_indices(m, BOTH_SAMPLE, 41)
    sub, sub_off = sub_batch(pats, off, both_ids)
    rc = oracle.revcomp_batch(sub, sub_off)
    rc_cnt = threaded(lambda a, b: oracle.count_sa(text, sa, rc[int(sub_off[a]):int(sub_off[b])],
                                                   (sub_off[a:b + 1] - sub_off[a]).astype(np.uint64)),
                      both_ids.size, threads)
    return {
        "workload": "QuadFm count, text 2^26 chars (20% planted repeats, 300-5000 long, 2% substitutions), "
                    "10^7 patterns 16..150 (even: sampled with 1% substitutions, odd: random); "
                    "workloads.fm_inputs()",
        "n": int(text.size), "patterns": int(m),
        "sa_uint32_sha256": sha(sa, "<u4"),
        "sa_first": [int(x) for x in sa[:8]],
        "counts_uint64_sha256": sha(cnt, "<u8"),
        "counts_sum": int(cnt.sum()), "counts_zero": int((cnt == 0).sum()),
        "counts_first": [int(x) for x in cnt[:16]],
        "revcomp_sample": {"ids": "workloads.sample_indices(patterns, 100000, 41)", "size": int(both_ids.size),
                           "counts_uint64_sha256": sha(rc_cnt, "<u8"), "counts_sum": int(rc_cnt.sum()),
                           "counts_first": [int(x) for x in rc_cnt[:16]]},
        "oracle": "oracle.suffix_array (comparison sort of the suffixes of T$), oracle.count_sa "
                  "(suffix-array interval by binary search), oracle.revcomp_batch",
        "seconds": {"suffix_array": round(t_sa, 1), "total": round(time.time() - t0, 1)},
    }


def serving_workload(threads: int) -> dict:
    t0 = time.time()
    text, pats, off, first = workloads.serving_inputs(SERVE_REQUESTS, 28)
    npat = int(first[-1])
    ids = workloads.sample_indices(npat, SERVE_SAMPLE, 43)
    sub, sub_off = sub_batch(pats, off, ids)
    cnt = threaded(lambda a, b: oracle.count_brute_batch(text, sub[int(sub_off[a]):int(sub_off[b])],
                                                         (sub_off[a:b + 1] - sub_off[a]).astype(np.uint64)),
                   ids.size, threads)
    return {
        "workload": "QuadFm serving, text 2^28 chars (same generator), the first 256 requests of "
                    "workloads.serving_inputs(256, 28): 1..4096 patterns each, lengths 16..250",
        "n": int(text.size), "requests": SERVE_REQUESTS, "patterns": npat,
        "sample_ids": [int(x) for x in ids], "sample_counts": [int(x) for x in cnt],
        "oracle": "oracle.count_brute_batch (direct comparison at every text position)",
        "seconds": round(time.time() - t0, 1),
    }


def main():
    threads = os.cpu_count() or 1
    which = sys.argv[1:] or ["count", "serving"]
    for w in which:
        d = count_workload(threads) if w == "count" else serving_workload(threads)
        d["written_by"] = "tests/golden/make_fm_full.py (oracle only)"
        name = "fm_full_2p26_1e7.json" if w == "count" else "fm_serving_2p28.json"
        (HERE / name).write_text(json.dumps(d, indent=1) + "\n")
        print(name, json.dumps({k: v for k, v in d.items() if k not in ("sample_ids", "sample_counts")}), flush=True)


if __name__ == "__main__":
    main()
