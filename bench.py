#!/usr/bin/env python3
"""Benchmark of the rank / QuadFm hot path on GB300.

Headline workload: BiRank (sigma 2) over n = 2^34 i.i.d. bits (p = 0.5),
2^28 uint64 queries uniform in [0, n], rank(q) into uint64 outputs; a step is
one qr_rank call over the whole batch.  The JSON line also carries the other
rows of the hot path measured in the same run (``extra``): sorted queries,
density 0.01, an L2-resident 2^26-bit text, QuadRank rank with random symbols
and rank_4 over 2^32 DNA chars, and QuadFm counts.

``--impl reference`` times the CPU oracle (the only comparison program this
project has) on a bounded sample of the same workload.

Multi-GPU: one process per GPU; each rank holds its own index and answers its
own 2^28 queries (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "rank Gqueries/s and % of HBM random-access roofline; QuadFm patterns/s"
B2 = 496
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- environment
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def to_dev_u64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def time_launches(fn, steps, stream):
    """Run fn() `steps` times; CUDA events on `stream` around each launch.
    Returns (total ms, list of per-launch ms)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in evs]


def barrier_sync(ws):
    import torch
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def traffic_record(kernel: str):
    """DRAM bytes per unit of a kernel from a committed ncu summary, if the
    kernel's sources have not changed since the capture."""
    import hashlib
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text()).get(kernel)
    if not d:
        return None
    h = hashlib.sha256()
    for f in d["sources"]:
        h.update((ROOT / f).read_bytes())
    if h.hexdigest() != d["sha256"]:
        return None
    return d


# ---------------------------------------------------------------- workloads
def birank_workload(n, m, seed_id, p=0.5, sorted_q=False):
    from paper_2602_04103_gb300 import synth
    base = synth.base_seed(seed_id)
    text = synth.bits(synth.substream(base, 1), n, p)
    q = synth.queries(synth.substream(base, 2), n, m)
    if sorted_q:
        q.sort()
    return text, q


def run_ours(args):
    import torch
    from paper_2602_04103_gb300 import capi

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = 1 << args.log_n
    m = 1 << args.log_m
    t_gen = time.time()
    # every rank answers its own batch (seed offset by rank): weak scaling
    text, q = birank_workload(n, m, 2 + 100 * rank)
    log(f"[bench] generated n=2^{args.log_n} bits, m=2^{args.log_m} queries in {time.time() - t_gen:.1f}s")
    d_text = to_dev_u64(text)
    idx = capi.qr_build(d_text, n, 2)
    del d_text
    if args.tune:
        capi.qr_set_tuning(idx, *args.tune)
    tuning = capi.qr_get_tuning(idx)
    dq = to_dev_u64(q)
    out = torch.empty_like(dq)

    def step():
        capi.qr_rank(idx, dq, 1, out)

    for _ in range(args.warmup):
        step()
    barrier_sync(ws)
    with ClockSampler(local) as clk:
        total_ms, per = time_launches(step, args.steps, stream)
        barrier_sync(ws)
    total_ms = max_over_ranks(total_ms, ws)
    status = capi.qr_status(idx)
    assert status == 0, f"device status {status}"
    value = ws * m * args.steps / (total_ms * 1e-3) / 1e9
    avg_ms = float(np.mean(per))
    bytes_per_q = 64 + 8 + 8
    achieved = bytes_per_q * m / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    tr = traffic_record("birank_rank")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": (round(tr["bytes_per_query"] * m) if tr else None),
                "peak_kind": f"of {peak_kind}",
                "algorithmic_bytes_per_query": bytes_per_q,
                "kernel": "rank_kernel<K,LOAD,kBiScalar>"}

    # end to end through the public API with host buffers
    qh = torch.from_numpy(q.view(np.int64)).pin_memory()
    oh = torch.empty(m, dtype=torch.int64).pin_memory()

    def e2e_step():
        capi.qr_rank_host(idx, qh, 1, oh)

    e2e_step()
    barrier_sync(ws)
    e_ms, _ = time_launches(e2e_step, max(1, min(args.steps, 3)), stream)
    e_ms = max_over_ranks(e_ms, ws)
    e_steps = max(1, min(args.steps, 3))
    e2e_val = ws * m * e_steps / (e_ms * 1e-3) / 1e9
    chunks = (m + (1 << 22) - 1) >> 22
    # spot check of the e2e output against the device output
    torch.cuda.synchronize()
    assert np.array_equal(oh[:1 << 16].numpy(), out[:1 << 16].cpu().numpy())

    extra = {}
    if not args.no_extra and rank == 0:
        idx.free()
        del dq, out, qh, oh
        torch.cuda.empty_cache()
        extra = run_extras(args)

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gqueries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"BiRank sigma=2 rank(q), n=2^{args.log_n} i.i.d. bits p=0.5, 2^{args.log_m} "
                               f"uniform uint64 queries per GPU", "n_bits": n, "queries_per_gpu": m,
                   "layout": "BiRank16 (3.28% overhead)", "tuning": tuning,
                   "l2": "inputs larger than L2 (2 GiB queries, 2.2 GB index)", "parallelism": f"replica x{ws}"},
        "roofline": roofline,
        "e2e": {"value": round(e2e_val, 3), "unit": "Gqueries/s", "h2d_bytes_per_step": 8 * m,
                "d2h_bytes_per_step": 8 * m, "api": "qr_rank_host (pinned host buffers, chunked pipeline)"},
        "gpu_launches": args.steps,
        "gpu_launches_e2e_per_step": chunks,
        "clocks": clocks,
    }
    if extra:
        line["extra"] = extra
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, n, text, q)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_extras(args):
    """Other rows of the hot path, each timed with CUDA events (L2 flushed by
    inputs larger than L2 unless stated)."""
    import torch
    from paper_2602_04103_gb300 import capi
    out = {}
    stream = torch.cuda.current_stream()
    peak, _ = peaks()
    m = 1 << args.log_m

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        _, per = time_launches(fn, reps, stream)
        return float(np.mean(per))

    # BiRank: sorted queries, density 0.01, L2-resident text
    for name, log_n, p, srt in [("birank_sorted", args.log_n, 0.5, True), ("birank_p001", args.log_n, 0.01, False),
                                ("birank_l2_resident_2^26", 26, 0.5, False)]:
        n = 1 << log_n
        text, q = birank_workload(n, m, 12, p=p, sorted_q=srt)
        idx = capi.qr_build(to_dev_u64(text), n, 2)
        del text
        dq = to_dev_u64(q)
        o = torch.empty_like(dq)
        ms = timed(lambda: capi.qr_rank(idx, dq, 1, o))
        info = capi.qr_info(idx)
        gq = m / (ms * 1e-3) / 1e9
        bpq = 16 + (64 if not srt and log_n > 27 else (info["bytes_blocks"] + info["bytes_super"]) / m)
        out[name] = {"Gq_s": round(gq, 3), "ms": round(ms, 3), "algorithmic_bytes_per_query": round(bpq, 2),
                     "roofline_frac": round(gq * bpq / peak, 4)}
        idx.free()
        del dq, o
        torch.cuda.empty_cache()
        log(f"[bench] {name}: {gq:.2f} Gq/s")

    # QuadRank over 2^32 uniform DNA chars: rank(q, c) with random c, and rank_4
    from paper_2602_04103_gb300 import synth
    n4 = 1 << args.log_n4
    base = synth.base_seed(3)
    t4 = synth.dna_uniform(synth.substream(base, 1), n4)
    q4 = synth.queries(synth.substream(base, 2), n4, m)
    c4 = synth.symbols(synth.substream(base, 3), m, 4)
    idx4 = capi.qr_build(to_dev_u64(t4), n4, 4)
    del t4
    dq = to_dev_u64(q4)
    dc = torch.from_numpy(c4).cuda()
    o = torch.empty_like(dq)
    ms = timed(lambda: capi.qr_rank_c(idx4, dq, dc, o))
    gq = m / (ms * 1e-3) / 1e9
    out["quadrank_rank_random_c"] = {"Gq_s": round(gq, 3), "ms": round(ms, 3), "algorithmic_bytes_per_query": 81,
                                     "roofline_frac": round(gq * 81 / peak, 4)}
    del o
    o4 = torch.empty((m, 4), dtype=torch.int64, device="cuda")
    ms = timed(lambda: capi.qr_rank4(idx4, dq, o4))
    gq = m / (ms * 1e-3) / 1e9
    out["quadrank_rank4"] = {"Gq_s": round(gq, 3), "ms": round(ms, 3), "algorithmic_bytes_per_query": 104,
                             "roofline_frac": round(gq * 104 / peak, 4)}
    idx4.free()
    del dq, dc, o4
    torch.cuda.empty_cache()
    log(f"[bench] quadrank: {out['quadrank_rank_random_c']['Gq_s']} / {out['quadrank_rank4']['Gq_s']} Gq/s")
    return out


def cpu_baseline(args, n, text, q):
    """The oracle as it stands, on a bounded sample of the workload: the
    sweep answers a sample of the same queries over the full text."""
    import oracle
    sample = q[: 1 << args.cpu_log_sample].copy()
    t0 = time.perf_counter()
    _, rc = oracle.rank(text, n, 2, sample, 1)
    dt = time.perf_counter() - t0
    return {"value": round(sample.size / dt / 1e9, 6), "unit": "Gqueries/s", "cores": 1, "kind": "oracle",
            "sample": f"first 2^{args.cpu_log_sample} of the queries over the full 2^{args.log_n}-bit text "
                      f"(sort + one linear sweep), {dt:.1f}s"}


def run_reference(args):
    """The CPU oracle as the reference arm: each step answers a bounded sample
    of the workload's queries over the full text."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n = 1 << args.log_n
    m = 1 << args.log_m
    text, q = birank_workload(n, m, 2)
    sample = q[: 1 << args.cpu_log_sample].copy()
    for _ in range(args.warmup):
        oracle.rank(text, n, 2, sample[: 1 << 16], 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rank(text, n, 2, sample, 1)
    dt = time.perf_counter() - t0
    value = args.steps * sample.size / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gqueries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"BiRank sigma=2 rank(q), n=2^{args.log_n} i.i.d. bits p=0.5, 2^{args.log_m} "
                                   f"uniform uint64 queries per GPU", "n_bits": n, "queries_per_gpu": m},
            "cpu_baseline": {"value": round(value, 6), "unit": "Gqueries/s", "cores": 1, "kind": "oracle",
                             "sample": f"2^{args.cpu_log_sample} of the queries per step over the full text"},
            "e2e": {"value": round(value, 6), "unit": "Gqueries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log-n", type=int, default=34)
    ap.add_argument("--log-m", type=int, default=28)
    ap.add_argument("--log-n4", type=int, default=32)
    ap.add_argument("--cpu-log-sample", type=int, default=22)
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tune", type=int, nargs=4, metavar=("K", "THREADS", "LOAD", "GRID"))
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("[bench] warmup raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
