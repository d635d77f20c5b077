"""Write fm_work_2p26_1e7.json: LF-step statistics of the QuadFm count workload
(2^26-char text with planted repeats, patterns of length 16..150, half
sampled with 1% substitutions), computed by the oracle only.

The count-only search (QuadRank paper, App. D) spends one LF step -- two rank
queries -- per pattern character after the 8-character table lookup while the
interval is non-empty; oracle.fm_steps counts those steps from the suffix
array of T$.  The benchmark multiplies the mean by the number of patterns to
get the rank queries (and bytes) one launch performs.

Run:  python tests/golden/make_fm_work.py   (about two minutes on one core)
"""
import json
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2602_04103_gb300 import synth  # noqa: E402

LOG_N = 26
M_ALL = 10_000_000
M_SAMPLE = 1_000_000


def main():
    base = synth.base_seed(4)
    t0 = time.time()
    text = synth.fm_text(synth.substream(base, 1), 1 << LOG_N)
    pats, off = synth.patterns(synth.substream(base, 5), text, M_ALL, 16, 150, 0.01)
    sa = oracle.suffix_array(text)
    # the first M_SAMPLE patterns of the workload (even = sampled, odd = random)
    sub_off = off[: M_SAMPLE + 1]
    total, steps = oracle.fm_steps(text, sa, pats, sub_off, k=8)
    lens = (sub_off[1:] - sub_off[:-1]).astype("int64")
    out = {
        "workload": "QuadFm count, text 2^26 chars (20% planted repeats, 300-5000 long, 2% substitutions), "
                    "patterns 16..150 (even: sampled with 1% substitutions, odd: random)",
        "seed_base": base, "log_n": LOG_N, "patterns_total": M_ALL, "patterns_sampled": M_SAMPLE,
        "lf_steps_sampled": int(total), "mean_lf_steps": total / M_SAMPLE,
        "mean_lf_steps_sampled_patterns": float(steps[0::2].mean()),
        "mean_lf_steps_random_patterns": float(steps[1::2].mean()),
        "mean_pattern_length": float(lens.mean()),
        "seconds": round(time.time() - t0, 1),
        "written_by": "tests/golden/make_fm_work.py (oracle only)",
    }
    (Path(__file__).parent / "fm_work_2p26_1e7.json").write_text(json.dumps(out, indent=1) + "\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
