#!/usr/bin/env python3
"""Benchmark of the rank / QuadFm hot path on GB300.

Headline (the workload the metric is quoted on): BiRank (sigma 2) over
n = 2^34 i.i.d. bits (p = 0.5), 2^28 uint64 queries uniform in [0, n],
rank(q) into uint64 outputs.  A step is one qr_rank call over the whole
batch, on an index built by the tuned build (every layout within the space
budget, autotuned, fastest kept).  The line also carries, measured in the
same run: the GPU's random 32-byte request ceiling (gather probe), the
end-to-end rate through the host-buffer API, and under ``extra`` the other
rows of the hot path (sorted queries, density 0.01, an L2-resident text,
QuadRank rank / rank_4 over 2^32 chars, QuadFm counts: persistent vs
per-step launches).

``--impl reference`` times the CPU oracle on a bounded sample of the same
workload (this project has no other comparison program).

Multi-GPU: one process per GPU, each holding its own index and answering its
own 2^28 queries (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
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
FALLBACK_HBM_GBS = 6800.0
CHUNK_HOST = 1 << 23  # queries per chunk of the host-buffer pipeline (qr_rank_host)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return float(json.loads(p.read_text())["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.lines = gpu_index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
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


def dev_u64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def time_launches(fn, steps, stream):
    """fn() `steps` times with CUDA events on `stream` around each call.
    Returns (total ms, per-call ms)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in evs]


def best_ms(fn, stream, reps=3):
    fn()
    _, per = time_launches(fn, reps, stream)
    return float(np.median(per))


def host_copy_bound(qh, oh, dev_out, stream, reps: int = 2):
    """The e2e path's own ceiling on this host: the pinned query buffer copied
    in and the result buffer copied out at once, on two streams, as the
    pipeline overlaps them; 16 bytes per query cross the link."""
    import torch
    d_in = torch.empty_like(dev_out)
    s2 = torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def both():  # the two copies start together, the next pair after both end
        s2.wait_stream(stream)
        with torch.cuda.stream(stream):
            d_in.copy_(qh, non_blocking=True)
        with torch.cuda.stream(s2):
            oh.copy_(dev_out, non_blocking=True)
        stream.wait_stream(s2)

    both()  # untimed: first copies into fresh buffers run several times slower
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        both()
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    gbs = reps * (qh.numel() + oh.numel()) * 8 / (ms * 1e-3) / 1e9
    del d_in
    return {"h2d_plus_d2h_GB_s": round(gbs, 1), "Gq_s": round(gbs / 16, 3)}


def barrier_sync(ws):
    import torch
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """Largest x over the ranks (the slowest rank's timed region)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def traffic_record(kernel: str):
    """DRAM bytes per query of a kernel from the committed ncu summary, if the
    kernel's sources are unchanged since the capture (else None)."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text()).get(kernel)
    if not d:
        return None
    h = hashlib.sha256()
    for f in d["sources"]:
        h.update((ROOT / f).read_bytes())
    return d if h.hexdigest() == d["sha256"] else None


LAYOUT_NAMES_BI = {0: "BiRank16 (3.28% overhead)", 1: "BiRank16x2 sector layout (6.72% overhead)",
                   2: "BiRank16 on 128-byte lines (1.69% overhead)", 3: "BiRank32 (6.67% overhead)",
                   4: "BiRank32x2 (14.3% overhead)"}


def bytes_per_query(sigma: int, layout: int, load_mode: int, rank4: bool = False, per_query_c: bool = False):
    """Algorithmic bytes of one query: the index bytes it must read (the
    32-byte half-line of the sector layout and of BiRank32x2, the 64-byte line
    of the paper layout and of BiRank32 / QuadRank32 / QuadRank24_8, the
    128-byte line of the line layout) + the 8-byte query + the result (8, or 32
    for rank_4) + 1 byte of symbol when symbols are per query."""
    index = {0: 64, 1: 32, 2: 128, 3: 64, 4: 32, 5: 64}[layout]
    return index + 8 + (32 if rank4 else 8) + (1 if per_query_c else 0)


def requests_per_query(sigma: int, layout: int, load_mode: int) -> float:
    """Random DRAM requests of one uniform query (superblock entries are
    L2-resident): the sector and 128-byte line layouts issue one request per
    query, and so does the paper layout's pair-cooperative load mode 4 (the two
    lanes' halves of a line in one instruction); load modes 1 and 3 read one
    sector below the block middle and two above it, modes 0 and 2 two."""
    if layout in (1, 2, 3, 4, 5) or load_mode == 4:
        return 1.0
    if load_mode in (0, 2):
        return 2.0
    lower = 240 / 496 if sigma == 2 else 96 / 224
    return lower + 2 * (1 - lower)


REGION_TILE, REGION_COUNT = 8192, 256
REGION_PASSES = ("sort", "rank", "unsort")
REGION_KERNELS = {"sort": "region_sort_tma<VEC>", "rank": "region_rank<SECTOR,QUAD,VEC,MODE>",
                  "unsort": "region_unsort (rank_4: region_unsort4)"}


def region_pass_bytes(m: int, index_bytes: int, per_query_c: bool = False, rank4: bool = False) -> dict:
    """Algorithmic DRAM bytes per query of each region-batching pass: the
    query word (and symbol) read once; a 4-byte key and a 2-byte index inside
    the tile written by the sort; the 4-byte segment entries (one per region
    and tile of 8192 queries) written twice by the sort (region-major for the
    rank pass, tile-major for the unsort) and read once by each later pass;
    the key read and the low 32 bits of the result written back by the rank
    pass (rank_4: the low 32 bits of the four counts, 16 bytes, written in
    sorted order); key (rank_4: the 16 bytes) and index read and the 8-byte
    result (rank_4: the 32-byte row) written by the unsort; the index read
    once per batch in the rank pass."""
    seg = 4.0 * REGION_COUNT / REGION_TILE
    sym = 1.0 if per_query_c else 0.0
    if rank4:
        return {"sort": 8 + sym + 6 + 2 * seg, "rank": 4 + 16 + seg + index_bytes / m, "unsort": 16 + 2 + seg + 32}
    return {"sort": 8 + sym + 6 + 2 * seg, "rank": 4 + 4 + seg + index_bytes / m, "unsort": 6 + seg + 8}


def region_passes(idx, step, m, index_bytes, per_query_c=False, rank4=False):
    """Per-pass times of a region-batched call (CUDA events the library
    records between its passes, median of 3 calls) and the passes' bytes."""
    from paper_2602_04103_gb300 import capi
    capi.qr_region_timing(idx, True)
    runs = []
    for _ in range(3):
        step()
        runs.append(capi.qr_region_timing(idx, True, read=True))
    capi.qr_region_timing(idx, False)
    pass_ms = {p: float(np.median([r[i] for r in runs])) for i, p in enumerate(REGION_PASSES)}
    return pass_ms, region_pass_bytes(m, index_bytes, per_query_c, rank4)


def region_roofline(idx, step, m, index_bytes, avg_ms, peak, peak_kind, stream, per_query_c=False, rank4=False,
                    traffic_key="birank_region"):
    """Roofline of the dominant pass of a region-batched step."""
    pass_ms, pbytes = region_passes(idx, step, m, index_bytes, per_query_c, rank4)
    dom = max(pass_ms, key=pass_ms.get)
    achieved = pbytes[dom] * m / (pass_ms[dom] * 1e-3) / 1e9
    tr = traffic_record(f"{traffic_key}_{dom}")
    step_bytes = sum(pbytes.values())
    passes = list(REGION_PASSES)
    # under the automatic rule every step also launches the probe, the direct
    # kernel (which returns at once when the probe picks region batching)
    # and the kernel of the region bases
    launches = len(passes) + 3
    return ({"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
             "frac": round(achieved / peak, 4), "traffic": round(tr["bytes_per_query"] * m) if tr else None,
             "peak_kind": f"of {peak_kind} (copy bandwidth)", "kernel": REGION_KERNELS[dom],
             "algorithmic_bytes_per_query": round(pbytes[dom], 3), "queries_per_launch": m,
             "passes_ms": {p: round(pass_ms[p], 4) for p in passes},
             "passes_bytes_per_query": {p: round(pbytes[p], 3) for p in passes},
             "passes_frac": {p: round(pbytes[p] * m / (pass_ms[p] * 1e-3) / 1e9 / peak, 4) for p in passes},
             "step_bytes_per_query": round(step_bytes, 3),
             "step_achieved_GB_s": round(step_bytes * m / (avg_ms * 1e-3) / 1e9, 1),
             "step_frac": round(step_bytes * m / (avg_ms * 1e-3) / 1e9 / peak, 4),
             "launches_per_step": launches}, launches)


# ---------------------------------------------------------------- our arm
def probe_ceiling(stream, quad128: bool = False):
    """Random 32-byte loads over a 4 GiB buffer: the GPU's random request rate.
    quad128: random 128-byte records, each read by the four lanes of a quad in
    one instruction (the access of the 128-byte line layout)."""
    import torch
    from paper_2602_04103_gb300 import capi
    nbytes, m = 4 << 30, 1 << 26
    buf = torch.empty(nbytes // 8, dtype=torch.int64, device="cuda")
    out = torch.empty(m, dtype=torch.int64, device="cuda")
    if quad128:
        ms = min(best_ms(lambda: capi.qr_probe_gather(buf, nbytes // 128, 128, m, 99, out, k, 256, load_bytes=128),
                         stream) for k in (1, 2))
    else:
        ms = best_ms(lambda: capi.qr_probe_gather(buf, nbytes // 32, 32, m, 99, out, 4, 256, load_bytes=32), stream)
    del buf, out
    torch.cuda.empty_cache()
    return m / (ms * 1e-3) / 1e9


def run_ours(args):
    import torch
    from paper_2602_04103_gb300 import capi, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    host = bind_to_gpu_node(local)
    stream = torch.cuda.current_stream()
    n, m = 1 << args.log_n, 1 << args.log_m
    t0 = time.time()
    text, q = workloads.birank_inputs(args.log_n, args.log_m, rank=rank)
    log(f"[bench] inputs n=2^{args.log_n} bits, m=2^{args.log_m} queries: {time.time() - t0:.1f}s")
    nan = float("nan")
    ceil32 = probe_ceiling(stream) if args.layout is None else nan
    ceil128 = probe_ceiling(stream, quad128=True) if args.layout is None else nan
    log(f"[bench] random request ceilings: 32-byte {ceil32:.2f} G/s, 128-byte quad {ceil128:.2f} G/s")
    dq = dev_u64(q)
    d_text = dev_u64(text)
    t0 = time.time()
    if args.layout is None:
        idx, layout, tuning = workloads.build_tuned(d_text, n, 2, dq, c=1)
    else:   # fixed layout and tuning (profiling runs): no autotuning launches
        layout = args.layout
        idx = capi.qr_build(d_text, n, 2, layout=layout)
        capi.qr_set_tuning(idx, args.tuning[0], args.tuning[1], args.tuning[2], 0)
        tuning = capi.qr_get_tuning(idx)
    t_tune = time.time() - t0
    del d_text
    torch.cuda.empty_cache()
    info = capi.qr_info(idx)
    log(f"[bench] tuned build: layout {layout}, {tuning} ({t_tune:.1f}s)")
    out = torch.empty_like(dq)
    ceiling = ceil128 if layout == 2 else ceil32
    plan = capi.qr_rank_plan(idx, m)
    log(f"[bench] batch path: {'region batching' if plan == capi.QR_BATCH_REGIONS else 'direct kernels'}")

    def step():
        capi.qr_rank(idx, dq, 1, out)

    # the sampler starts first, so that the timed steps follow the warm-up
    # steps without an idle gap (an idle GPU lowers its clocks)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        barrier_sync(ws)
        total_ms, per = time_launches(step, args.steps, stream)
        barrier_sync(ws)
    total_ms = max_over_ranks(total_ms, ws)
    assert capi.qr_status(idx) == 0
    value = ws * m * args.steps / (total_ms * 1e-3) / 1e9
    avg_ms = float(np.mean(per))
    peak, peak_kind = peaks()
    index_bytes = info["bytes_blocks"] + info["bytes_super"]
    rpq = requests_per_query(2, layout, tuning["load_mode"])
    if plan == capi.QR_BATCH_REGIONS:
        roofline, launches = region_roofline(idx, step, m, index_bytes, avg_ms, peak, peak_kind, stream)
        # the rank pass against the L2: its read requests per query (ncu, the
        # committed capture) at the pass's rate, over the random 32-byte
        # request rate of an L2-resident buffer (qr_probe_l2: 64-byte records
        # are two 32-byte loads)
        tr = traffic_record("birank_region_rank")
        if tr and "l2_read_requests_per_query" in tr:
            rec_s, _ = l2_probe(20 << 20, stream)
            rq = tr["l2_read_requests_per_query"] * m / (roofline["passes_ms"]["rank"] * 1e-3)
            roofline["rank_pass_l2_requests"] = {
                "requests_per_query": tr["l2_read_requests_per_query"], "G_requests_per_s": round(rq / 1e9, 1),
                "l2_probe_G_requests_per_s": round(2 * rec_s / 1e9, 1), "frac": round(rq / (2 * rec_s), 4)}
            if "l2_read_sectors_per_query" in tr:
                # the same in 32-byte sectors: a request of the key stream or
                # of a warp's coalesced loads carries several (the probe's
                # requests carry one each)
                sq = tr["l2_read_sectors_per_query"] * m / (roofline["passes_ms"]["rank"] * 1e-3)
                roofline["rank_pass_l2_requests"].update(
                    sectors_per_query=tr["l2_read_sectors_per_query"], G_sectors_per_s=round(sq / 1e9, 1),
                    frac_sectors=round(sq / (2 * rec_s), 4))
        # the direct kernels on the same index and queries, for comparison
        capi.qr_set_batch_mode(idx, capi.QR_BATCH_DIRECT)
        ms_d = best_ms(step, stream)
        capi.qr_set_batch_mode(idx, capi.QR_BATCH_AUTO)
        gq_d = m / (ms_d * 1e-3) / 1e9
        roofline["direct_path"] = {
            "Gq_s": round(gq_d, 3), "ms": round(ms_d, 3),
            "algorithmic_bytes_per_query": bytes_per_query(2, layout, tuning["load_mode"]),
            "random_requests_per_query": round(rpq, 3),
            "random_request_ceiling_G_per_s": round(ceiling, 2) if ceiling == ceiling else None,
            "frac_of_random_request_ceiling": round(gq_d * rpq / ceiling, 4) if ceiling == ceiling else None}
        log(f"[bench] direct kernels on the same batch: {gq_d:.2f} Gq/s")
    else:
        launches = 1
        bpq = bytes_per_query(2, layout, tuning["load_mode"])
        achieved = bpq * m / (avg_ms * 1e-3) / 1e9
        kname = {0: "birank_rank_paper", 1: "birank_rank_sector", 2: "birank_rank_line128", 3: "birank_rank_in32",
                 4: "birank_rank_in32x2"}[layout]
        tr = traffic_record(kname)
        gq_launch = m / (avg_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": round(tr["bytes_per_query"] * m) if tr else None,
                    "peak_kind": f"of {peak_kind} (copy bandwidth)",
                    "kernel": {0: "rank_kernel<K,LOAD,kBiScalar>", 1: "rank_sector_kernel<K,kBiScalar>",
                               2: "rank_line_kernel<K,kBiScalar>", 3: "rank_in32_kernel<K,kBiScalar,false>",
                               4: "rank_in32_kernel<K,kBiScalar,true>"}[layout],
                    "algorithmic_bytes_per_query": bpq, "queries_per_launch": m,
                    "random_requests_per_query": round(rpq, 3),
                    "random_request_ceiling_G_per_s": round(ceiling, 2) if ceiling == ceiling else None,
                    "random_request_ceiling_kind": "128-byte quad-cooperative" if layout == 2 else "32-byte",
                    "frac_of_random_request_ceiling": round(gq_launch * rpq / ceiling, 4) if ceiling == ceiling
                    else None}

    # end to end through the public host-buffer API (H2D + kernels + D2H)
    qh = torch.from_numpy(q.view(np.int64)).pin_memory()
    oh = torch.empty(m, dtype=torch.int64).pin_memory()

    def e2e_step():
        capi.qr_rank_host(idx, qh, 1, oh)

    # the first calls on freshly pinned buffers run 4-8x slower on GB300 (87,
    # 112, 53 ms against a steady 13.4 ms, measured): the warm-up takes the
    # same W steps as the kernel timing, at least three
    for _ in range(max(3, args.warmup)):
        e2e_step()
    barrier_sync(ws)
    e_steps = max(1, min(args.steps, 5))
    e_ms, _ = time_launches(e2e_step, e_steps, stream)
    e_ms = max_over_ranks(e_ms, ws)
    e2e_val = ws * m * e_steps / (e_ms * 1e-3) / 1e9
    torch.cuda.synchronize()
    assert np.array_equal(oh[: 1 << 16].numpy(), out[: 1 << 16].cpu().numpy())
    copy_bound = host_copy_bound(qh, oh, out, stream)

    extra = {}
    if not args.no_extra and rank == 0:
        extra = run_extras(args, idx, layout, tuning, dq, out, stream, peak)
    idx.free()
    del dq, out, qh, oh
    torch.cuda.empty_cache()
    if not args.no_extra and rank == 0:
        extra.update(run_extras_other(args, stream, peak))

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gqueries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"BiRank sigma=2 rank(q), n=2^{args.log_n} i.i.d. bits p=0.5, 2^{args.log_m} "
                               f"uniform uint64 queries per GPU",
                   "n_bits": n, "queries_per_gpu": m,
                   "layout": LAYOUT_NAMES_BI[layout],
                   "index_bytes": index_bytes, "tuning": tuning,
                   "batch_path": "region batching (tiles of 8192 queries sorted by 256 text regions, answered "
                                 "region after region from L2, results put back in query order)"
                   if plan == capi.QR_BATCH_REGIONS else "direct kernels (one line load per query)",
                   "tuned_build_s": round(t_tune, 2),
                   "l2": "inputs larger than L2 (2 GiB queries, 2.3 GB index; L2 129 MB)",
                   "parallelism": f"independent replica per GPU x{ws}", "host": host},
        "roofline": roofline,
        "e2e": {"value": round(e2e_val, 3), "unit": "Gqueries/s", "h2d_bytes_per_step": 8 * m,
                "d2h_bytes_per_step": 8 * m,
                "api": "qr_rank_host: pinned host q/out, chunks of 2^23 on four streams",
                "copy_bound": dict(copy_bound, frac=round(e2e_val / (ws * copy_bound["Gq_s"]), 4))},
        "gpu_launches": args.steps * launches,
        "gpu_launches_e2e_per_step": (m + CHUNK_HOST - 1) // CHUNK_HOST,
        "clocks": clk.summary(),
    }
    if extra:
        line["extra"] = extra
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, n, text, q)
        if not args.no_extra:
            line.setdefault("extra", {})["cpu_baseline_qfm_count"] = cpu_baseline_fm(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_extras(args, idx, layout, tuning, dq, out, stream, peak):
    """Rows that reuse the headline index: the same queries sorted."""
    import torch
    from paper_2602_04103_gb300 import capi
    m = dq.numel()
    res = {}
    qs = torch.sort(dq).values
    ms = best_ms(lambda: capi.qr_rank(idx, qs, 1, out), stream)
    info = capi.qr_info(idx)
    gq = m / (ms * 1e-3) / 1e9
    bpq = 16 + (info["bytes_blocks"] + info["bytes_super"]) / m   # every line once + q + out
    res["birank_sorted_queries"] = {"Gq_s": round(gq, 3), "ms": round(ms, 3),
                                    "algorithmic_bytes_per_query": round(bpq, 2),
                                    "roofline_frac": round(gq * bpq / peak, 4), "layout": layout}
    log(f"[bench] sorted: {gq:.2f} Gq/s")
    # latency mode: dependent queries (each position from the previous answer)
    res["birank_dependent_queries"] = dict(dependent_queries(idx, dq, stream), layout=layout,
                                           note="qr_rank_chain: each query position is derived from the previous answer")
    log(f"[bench] dependent: {res['birank_dependent_queries']}")
    return res


def dependent_queries(idx, dq, stream):
    """One chain of 2000 dependent queries (latency) and 2^20 chains of 64."""
    import torch
    from paper_2602_04103_gb300 import capi
    q0 = dq[: 1 << 20]
    o2 = torch.empty((q0.numel(), 2), dtype=torch.int64, device="cuda")
    steps1, stepsN = 2000, 64
    ms1 = best_ms(lambda: capi.qr_rank_chain(idx, q0[:1], steps1, 1, o2), stream)
    msN = best_ms(lambda: capi.qr_rank_chain(idx, q0, stepsN, 1, o2), stream)
    return {"one_chain_ns_per_query": round(ms1 * 1e6 / steps1, 1),
            "chains_2^20_Gq_s": round(q0.numel() * stepsN / (msN * 1e-3) / 1e9, 3)}


def run_layouts(args, stream):
    """The space-time front: every layout of BiRank (n = 2^34) and QuadRank
    (n = 2^32, rank with random symbols and rank_4), each autotuned on the
    first 2^24 queries, timed on the full 2^28."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    m = 1 << args.log_m
    names = {0: "paper (BiRank16 / QuadRank16)", 1: "sector (BiRank16x2 / 4-delta sectors)", 2: "128-byte lines",
             3: "32-bit inline (BiRank32 / QuadRank32)", 4: "32-bit inline x2 (BiRank32x2)",
             5: "QuadRank24_8"}
    res = {"birank": {}, "quadrank": {}}
    text, q = workloads.birank_inputs(args.log_n, args.log_m)
    dq, o = dev_u64(q), None
    o = torch.empty_like(dq)
    dt = dev_u64(text)
    del text
    for layout in (0, 1, 2, 3, 4):
        idx = capi.qr_build(dt, 1 << args.log_n, 2, layout=layout)
        t = capi.qr_autotune(idx, dq[: 1 << 24], o, c=1)
        ms = best_ms(lambda: capi.qr_rank(idx, dq, 1, o), stream)
        info = capi.qr_info(idx)
        res["birank"][names[layout]] = {"Gq_s": round(m / (ms * 1e-3) / 1e9, 3), "tuning": t,
                                        "overhead_pct": round(100 * ((info["bytes_blocks"] + info["bytes_super"]) * 8
                                                                     / (1 << args.log_n) - 1), 3),
                                        "dependent": dependent_queries(idx, dq, stream)}
        idx.free()
    del dt, dq, o
    torch.cuda.empty_cache()
    t4, q4, c4 = workloads.quadrank_inputs(args.log_n4, args.log_m)
    dq, dc = dev_u64(q4), torch.from_numpy(c4).cuda()
    o = torch.empty_like(dq)
    o4 = torch.empty((m, 4), dtype=torch.int64, device="cuda")
    d4 = dev_u64(t4)
    del t4
    for layout in (0, 1, 2, 3, 5):
        idx = capi.qr_build(d4, 1 << args.log_n4, 4, layout=layout)
        t1 = capi.qr_autotune(idx, dq[: 1 << 24], o, c=dc[: 1 << 24])
        ms1 = best_ms(lambda: capi.qr_rank_c(idx, dq, dc, o), stream)
        t4r = capi.qr_autotune(idx, dq[: 1 << 24], o4, rank4=True)
        ms4 = best_ms(lambda: capi.qr_rank4(idx, dq, o4), stream)
        info = capi.qr_info(idx)
        res["quadrank"][names[layout]] = {
            "rank_Gq_s": round(m / (ms1 * 1e-3) / 1e9, 3), "rank4_Gq_s": round(m / (ms4 * 1e-3) / 1e9, 3),
            "overhead_pct": round(100 * ((info["bytes_blocks"] + info["bytes_super"]) * 8
                                         / (2 * (1 << args.log_n4)) - 1), 3)}
        idx.free()
    del d4, dq, dc, o, o4
    torch.cuda.empty_cache()
    res["random_request_ceilings_G_per_s"] = {"32-byte": round(probe_ceiling(stream), 3),
                                              "128-byte quad": round(probe_ceiling(stream, quad128=True), 3)}
    log("[bench] layouts: " + json.dumps(res))
    return {"layouts": res}


def run_extras_other(args, stream, peak):
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    res = {}
    m = 1 << args.log_m
    # BiRank p = 0.01 (full size) and an L2-resident 2^26-bit text
    for name, log_n, p in [("birank_p0.01", args.log_n, 0.01), ("birank_l2_resident_2^26", 26, 0.5)]:
        text, q = workloads.birank_inputs(log_n, args.log_m, p=p, workload=12)
        dq = dev_u64(q)
        idx, layout, tuning = workloads.build_tuned(dev_u64(text), 1 << log_n, 2, dq, c=1)
        del text
        o = torch.empty_like(dq)
        ms = best_ms(lambda: capi.qr_rank(idx, dq, 1, o), stream)
        gq = m / (ms * 1e-3) / 1e9
        bpq = bytes_per_query(2, layout, tuning["load_mode"]) if log_n > 27 else 16
        res[name] = {"Gq_s": round(gq, 3), "ms": round(ms, 3), "layout": layout, "tuning": tuning,
                     "algorithmic_bytes_per_query": bpq, "roofline_frac": round(gq * bpq / peak, 4)}
        log(f"[bench] {name}: {gq:.2f} Gq/s")
        idx.free()
        del dq, o
        torch.cuda.empty_cache()
    res.update(run_quadrank(args, stream, peak))
    res.update(run_layouts(args, stream))
    res.update(run_fm(args, stream))
    res.update(run_serving(args))
    return res


def run_quadrank(args, stream, peak):
    """QuadRank over 2^32 uniform DNA: rank(q, c) with random c, prefix_rank
    and rank_4, each on the layout the tuned build picks for it."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    res = {}
    m = 1 << args.log_m
    n4 = 1 << args.log_n4
    peak_kind = peaks()[1]
    t4, q4, c4 = workloads.quadrank_inputs(args.log_n4, args.log_m, "uniform")
    dq, dc = dev_u64(q4), torch.from_numpy(c4).cuda()
    d4 = dev_u64(t4)
    del t4
    idx4, layout4, tuning4 = workloads.build_tuned(d4, n4, 4, dq, c=dc)
    info = capi.qr_info(idx4)
    index_bytes = info["bytes_blocks"] + info["bytes_super"]
    o = torch.empty_like(dq)
    step = lambda: capi.qr_rank_c(idx4, dq, dc, o)  # noqa: E731
    ms = best_ms(step, stream)
    gq = m / (ms * 1e-3) / 1e9
    regions = capi.qr_rank_plan(idx4, m) == capi.QR_BATCH_REGIONS
    row = {"Gq_s": round(gq, 3), "ms": round(ms, 3), "layout": layout4, "tuning": tuning4,
           "batch_path": "regions" if regions else "direct"}
    if regions:
        row["roofline"], _ = region_roofline(idx4, step, m, index_bytes, ms, peak, peak_kind, stream,
                                             per_query_c=True, traffic_key="quadrank_region")
    else:
        bpq = bytes_per_query(4, layout4, tuning4["load_mode"], per_query_c=True)
        row.update(algorithmic_bytes_per_query=bpq, roofline_frac=round(gq * bpq / peak, 4))
    res["quadrank_rank_random_c"] = row
    # prefix_rank(q, 2): characters <= G before q, same index and queries
    ms = best_ms(lambda: capi.qr_prefix_rank(idx4, dq, 2, o), stream)
    res["quadrank_prefix_rank"] = {"Gq_s": round(m / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3), "layout": layout4,
                                   "batch_path": "regions" if capi.qr_rank_plan(idx4, m, 2) == capi.QR_BATCH_REGIONS
                                   else "direct"}
    idx4.free()
    del o
    torch.cuda.empty_cache()
    # rank_4 on the layout its own tuned build picks
    o4 = torch.empty((m, 4), dtype=torch.int64, device="cuda")
    idx4, layout_r4, tuning_r4 = workloads.build_tuned(d4, n4, 4, dq, rank4=True)
    info = capi.qr_info(idx4)
    index_bytes = info["bytes_blocks"] + info["bytes_super"]
    step4 = lambda: capi.qr_rank4(idx4, dq, o4)  # noqa: E731
    ms = best_ms(step4, stream)
    gq = m / (ms * 1e-3) / 1e9
    regions = capi.qr_rank_plan(idx4, m, 1) == capi.QR_BATCH_REGIONS
    row = {"Gq_s": round(gq, 3), "ms": round(ms, 3), "layout": layout_r4, "tuning": tuning_r4,
           "batch_path": "regions" if regions else "direct"}
    if regions:
        row["roofline"], _ = region_roofline(idx4, step4, m, index_bytes, ms, peak, peak_kind, stream, rank4=True,
                                             traffic_key="quadrank4_region")
        capi.qr_set_batch_mode(idx4, capi.QR_BATCH_DIRECT)
        ms_d = best_ms(step4, stream)
        capi.qr_set_batch_mode(idx4, capi.QR_BATCH_AUTO)
        row["direct_path"] = {"Gq_s": round(m / (ms_d * 1e-3) / 1e9, 3), "ms": round(ms_d, 3),
                              "algorithmic_bytes_per_query": bytes_per_query(4, layout_r4, tuning_r4["load_mode"],
                                                                             rank4=True)}
    else:
        bpq = bytes_per_query(4, layout_r4, tuning_r4["load_mode"], rank4=True)
        row.update(algorithmic_bytes_per_query=bpq, roofline_frac=round(gq * bpq / peak, 4))
    res["quadrank_rank4"] = row
    log(f"[bench] quadrank: {res['quadrank_rank_random_c']['Gq_s']} / {res['quadrank_rank4']['Gq_s']} Gq/s")
    idx4.free()
    del dq, dc, o4, d4
    torch.cuda.empty_cache()
    res["quadrank_gc_runs"] = run_quadrank_gc(args, stream)
    return res


def run_quadrank_gc(args, stream):
    """The second QuadRank text: GC 40 %, homopolymer runs of 10..1000 over 5 %
    of it; rank with random symbols and rank_4, each on its tuned layout."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    m = 1 << args.log_m
    n4 = 1 << args.log_n4
    t4, q4, c4 = workloads.quadrank_inputs(args.log_n4, args.log_m, "gc_runs")
    dq, dc = dev_u64(q4), torch.from_numpy(c4).cuda()
    d4 = dev_u64(t4)
    del t4
    row = {"text": "gc_runs: P(C) = P(G) = 0.2, P(A) = P(T) = 0.3, runs of one symbol (10..1000) over 5 %"}
    idx4, layout, _ = workloads.build_tuned(d4, n4, 4, dq, c=dc)
    o = torch.empty_like(dq)
    ms = best_ms(lambda: capi.qr_rank_c(idx4, dq, dc, o), stream)
    row["rank_random_c"] = {"Gq_s": round(m / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3), "layout": layout}
    idx4.free()
    del o
    o4 = torch.empty((m, 4), dtype=torch.int64, device="cuda")
    idx4, layout, _ = workloads.build_tuned(d4, n4, 4, dq, rank4=True)
    ms = best_ms(lambda: capi.qr_rank4(idx4, dq, o4), stream)
    row["rank4"] = {"Gq_s": round(m / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3), "layout": layout}
    idx4.free()
    del dq, dc, o4, d4
    torch.cuda.empty_cache()
    log(f"[bench] quadrank gc_runs: {row['rank_random_c']['Gq_s']} / {row['rank4']['Gq_s']} Gq/s")
    return row


def run_fm(args, stream, part="all"):
    """QuadFm count over the 2^26-char text, 10^7 patterns of length 16..150:
    one persistent launch vs one launch per search step; then locate and
    approximate counts.  part = "locate" or "approx" runs the persistent count
    and that row alone (few launches: profiling runs)."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    text, pats, off = workloads.fm_inputs(args.fm_log_n, args.fm_m)
    m = off.size - 1
    dt = torch.from_numpy(text).cuda()
    torch.cuda.synchronize()
    t0 = time.time()
    fidx = capi.qfm_build(dt, text.size)
    torch.cuda.synchronize()
    t_build = time.time() - t0
    info = capi.qfm_info(fidx)
    dp = torch.from_numpy(pats).cuda()
    doff = torch.from_numpy(off.view(np.int64)).cuda()
    o = torch.empty(m, dtype=torch.int64, device="cuda")
    ms_p = best_ms(lambda: capi.qfm_count(fidx, dp, doff, o), stream)
    ref = o.clone()
    if part != "all":
        res = {"qfm_count_persistent": {"patterns_per_s": round(m / (ms_p * 1e-3)), "ms": round(ms_p, 3)}}
        fidx.free()
        if part == "locate":
            res.update(fm_locate_row(dt, text.size, dp, doff, m, ref, ms_p, stream))
        else:
            res.update(fm_approx_row(dt, text.size, dp, doff, ref, stream))
        return res
    ms_s = best_ms(lambda: capi.qfm_count_stepwise(fidx, dp, doff, o), stream)
    assert torch.equal(ref, o)
    # both strands in one launch (the paper's read-counting benchmark counts each read forward
    # and reverse-complemented)
    o2 = torch.empty(2 * m, dtype=torch.int64, device="cuda")
    ms_b = best_ms(lambda: capi.qfm_count_ex(fidx, dp, doff, o2, capi.QFM_BOTH_STRANDS), stream)
    assert torch.equal(o2[:m], ref)
    assert capi.qfm_status(fidx) == 0
    res = {"qfm_count_persistent": {"patterns_per_s": round(m / (ms_p * 1e-3)), "ms": round(ms_p, 3)},
           "qfm_count_stepwise": {"patterns_per_s": round(m / (ms_s * 1e-3)), "ms": round(ms_s, 3)},
           "qfm_count_both_strands": {"reads_per_s": round(m / (ms_b * 1e-3)), "searches_per_s": round(2 * m / (ms_b * 1e-3)),
                                      "ms": round(ms_b, 3)},
           "qfm_speedup_persistent_vs_stepwise": round(ms_s / ms_p, 2),
           "qfm_build_s": round(t_build, 3), "qfm_index_bytes": info["bytes_rank"] + info["bytes_table"]}
    work = ROOT / "tests" / "golden" / "fm_work_2p26_1e7.json"
    if work.exists() and args.fm_log_n == 26 and args.fm_m == 10_000_000:
        w = json.loads(work.read_text())
        steps = w["mean_lf_steps"] * m
        res["qfm_count_persistent"]["lf_steps_per_s"] = round(steps / (ms_p * 1e-3))
        res["qfm_count_persistent"]["rank_queries_per_s"] = round(2 * steps / (ms_p * 1e-3))
        res["qfm_lf_steps_source"] = "oracle mean over the first 10^6 patterns (tests/golden/fm_work_2p26_1e7.json)"
        res["qfm_count_persistent"]["roofline"] = fm_roofline(steps / (ms_p * 1e-3),
                                                              info["bytes_rank"] + info["bytes_table"], stream)
    log(f"[bench] qfm: persistent {m / ms_p / 1e3:.1f} M/s, stepwise {m / ms_s / 1e3:.1f} M/s")
    fidx.free()
    res.update(fm_locate_row(dt, text.size, dp, doff, m, ref, ms_p, stream))
    res.update(fm_approx_row(dt, text.size, dp, doff, ref, stream))
    return res


def l2_probe(index_bytes, stream):
    """Random 64-byte record reads from an L2-resident buffer the size of
    the FM index: (records/s with 4 independent reads per thread and round at
    full occupancy, dependent record pairs/s at the count kernel's occupancy
    of 1024 threads per SM)."""
    import torch
    from paper_2602_04103_gb300 import capi
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nrec = max(1, index_bytes // 64)
    buf = torch.zeros(nrec * 8, dtype=torch.int64, device="cuda")
    n0, r0 = sms * 2048, 256
    n1, r1 = sms * 1024, 512
    out = torch.empty(max(n0, n1), dtype=torch.int64, device="cuda")
    ms0 = best_ms(lambda: capi.qr_probe_l2(buf, nrec, 0, n0, r0, 7, out), stream)
    ms1 = best_ms(lambda: capi.qr_probe_l2(buf, nrec, 1, n1, r1, 7, out), stream)
    del buf, out
    torch.cuda.empty_cache()
    return 4 * n0 * r0 / (ms0 * 1e-3), n1 * r1 / (ms1 * 1e-3)


# L2 bytes one rank query reads from a QuadRank16 line (Sec. 4): a position in
# the lower half (96 of the 224 characters) needs the line's first 32-byte
# sector (deltas and counted characters); one in the upper half (128 of 224)
# needs the 16 delta bytes and the second sector.  Uniform over a block:
QFM_RANK_L2_BYTES = (96 * 32 + 128 * (16 + 32)) / 224


def fm_roofline(lf_steps_per_s, index_bytes, stream):
    """The count kernel against the L2 ceiling.  An LF step takes two rank
    queries (the lo and hi ends), each reading QFM_RANK_L2_BYTES of its line
    from the L2-resident index: 82.3 algorithmic L2 bytes per step (the
    kernel fetches a half-line once when both ends fall in it, so it can
    read less).  The peak is the L2 probe's random-read rate over a buffer
    the size of the index, in bytes (64-byte records, two 32-byte sector
    loads each, four records in flight per thread)."""
    rec_s, pair_s = l2_probe(index_bytes, stream)
    step_bytes = 2 * QFM_RANK_L2_BYTES
    achieved = lf_steps_per_s * step_bytes / 1e9
    peak = rec_s * 64 / 1e9
    log(f"[bench] L2 probe: {rec_s / 1e9:.1f} G records/s, {pair_s / 1e9:.1f} G dependent pairs/s")
    return {"bound": "l2", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": "of measured (qr_probe_l2: random 64-byte records "
            "from an L2-resident buffer the size of the index, 4 independent reads in flight per thread)",
            "algorithmic_bytes_per_lf_step": round(step_bytes, 2), "lf_steps_per_s": round(lf_steps_per_s),
            "l2_records_per_s": round(rec_s), "l2_dependent_pairs_per_s": round(pair_s),
            "frac_of_dependent_pair_rate": round(lf_steps_per_s / pair_s, 4),
            "frac_two_64B_lines_per_step": round(lf_steps_per_s * 128 / (rec_s * 64), 4),
            "index_bytes": index_bytes}


def fm_policies(args, stream):
    """The count kernel under each L2 policy (1, 2, 0; two launches each, the
    second timed with CUDA events) on the count workload: the measurement
    behind the default policy."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    text, pats, off = workloads.fm_inputs(args.fm_log_n, args.fm_m)
    m = off.size - 1
    fidx = capi.qfm_build(torch.from_numpy(text).cuda(), text.size)
    dp = torch.from_numpy(pats).cuda()
    doff = torch.from_numpy(off.view(np.int64)).cuda()
    o = torch.empty(m, dtype=torch.int64, device="cuda")
    res, ref = {}, None
    for pol in (1, 2, 0):
        capi.qfm_set_policy(fidx, pol)
        capi.qfm_count(fidx, dp, doff, o)
        _, per = time_launches(lambda: capi.qfm_count(fidx, dp, doff, o), 1, stream)
        ref = o.clone() if ref is None else ref
        assert torch.equal(o, ref)
        res[f"policy_{pol}"] = {"ms": round(per[0], 3), "patterns_per_s": round(m / (per[0] * 1e-3))}
    fidx.free()
    return res


def fm_locate_row(dt, n, dp, doff, m, ref, ms_p, stream):
    """Locate every occurrence of all patterns on the same text indexed with
    suffix-array sampling factor 32 (count with intervals, scan, LF walks)."""
    import torch
    from paper_2602_04103_gb300 import capi
    sample = 32
    lidx = capi.qfm_build(dt, n, 0, sa_sample=sample)
    linfo = capi.qfm_info(lidx)
    occ = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    total = capi.qfm_locate(lidx, dp, doff, occ)
    pos = torch.empty(max(total, 1), dtype=torch.int64, device="cuda")
    ms_l = best_ms(lambda: capi.qfm_locate(lidx, dp, doff, occ, pos), stream)
    assert torch.equal(occ[1:] - occ[:-1], ref)
    assert capi.qfm_status(lidx) == 0
    row = {"patterns_per_s": round(m / (ms_l * 1e-3)), "occurrences": total,
           "occurrences_per_s": round(total / (ms_l * 1e-3)), "ms": round(ms_l, 3),
           "ms_beyond_count": round(ms_l - ms_p, 3), "sa_sample": sample, "bytes_locate": linfo["bytes_locate"],
           "note": "whole qfm_locate call: count with intervals, scan, total read-back, one thread per "
                   "occurrence walking at most 31 LF steps"}
    log(f"[bench] qfm locate: {total} occurrences in {ms_l:.3f} ms")
    lidx.free()
    return {"qfm_locate": row}


def fm_approx_row(dt, n, dp, doff, ref, stream):
    """Approximate counts (at most k substitutions) on leading subsets of the
    patterns: rank_4 of both interval ends at every search node."""
    import torch
    from paper_2602_04103_gb300 import capi
    fidx = capi.qfm_build(dt, n)
    rows = {}
    for k, mk in [(0, 10 ** 6), (1, 10 ** 6), (2, 10 ** 5)]:
        mk = min(mk, ref.numel())
        ok = doff[: mk + 1]
        oa = torch.empty(mk, dtype=torch.int64, device="cuda")
        ms_a = best_ms(lambda: capi.qfm_count_approx(fidx, dp, ok, k, oa), stream)
        if k == 0:
            assert torch.equal(oa, ref[:mk])
        rows[f"k={k}"] = {"patterns": mk, "patterns_per_s": round(mk / (ms_a * 1e-3)), "ms": round(ms_a, 3),
                          "mean_count": round(float(oa.double().mean()), 3),
                          "kernel": "count_persistent (exact)" if k == 0 else "count_approx_kernel"}
        log(f"[bench] qfm approx k={k}: {mk / ms_a / 1e3:.2f} M patterns/s")
    assert capi.qfm_status(fidx) == 0
    fidx.free()
    return {"qfm_count_approx": rows}


def run_serving(args):
    """QuadFm serving over a 2^28-char index.  Arms: the continuous-batching
    server (4 slots, requests packed into shared batches); the same server with
    one request per batch on 4 slots (overlap without batching) and on 1 slot
    (serialised), the latter also with a spinning completion poll instead of
    the 20 us sleep; and a plain loop of qfm_count calls (copy in, count, copy
    out, wait) timed with CUDA events.  Each arm: closed-loop capacity, then
    Poisson arrivals at fractions of its own capacity (p50 / p99 latency at
    loads it sustains); the batching server also at 0.5..1.2x of its capacity."""
    import torch
    from paper_2602_04103_gb300 import capi, workloads
    text, pats, off, first = workloads.serving_inputs(args.serve_requests, args.serve_log_n)
    nreq = first.size - 1
    npat = int(first[-1])
    # the request trace lives in page-locked host memory (as an input reader
    # would keep it), so batches of back-to-back requests copy straight from it
    pats_t = torch.from_numpy(pats).pin_memory()
    pats = pats_t.numpy()
    off = torch.from_numpy(off.view(np.int64)).pin_memory().numpy().view(np.uint64)
    fidx = capi.qfm_build(torch.from_numpy(text).cuda(), text.size)
    del text
    res = {"serving_index_chars": 1 << args.serve_log_n, "serving_requests": nreq, "serving_patterns": npat,
           "serving_mean_patterns_per_request": round(npat / nreq, 1)}
    modes = {"batched": dict(slots=4), "per_request_4_slots": dict(slots=4, max_requests_per_batch=1),
             "per_request": dict(slots=1, max_requests_per_batch=1),
             "per_request_spin_poll": dict(slots=1, max_requests_per_batch=1, poll_us=0)}
    if args.serve_stream_calls:
        modes["batched_stream_calls"] = dict(slots=4, use_graph=0)
    ref = None
    rng = np.random.default_rng(55)

    def summary(mk, lat_us, st=None, gpu_us=None):
        d = {"patterns_per_s": round(npat / mk), "makespan_s": round(mk, 4),
             "p50_ms": round(float(np.percentile(lat_us, 50)) / 1e3, 3),
             "p99_ms": round(float(np.percentile(lat_us, 99)) / 1e3, 3)}
        if st is not None:
            d["mean_requests_per_batch"] = round(st["mean_requests_per_batch"], 2)
        if gpu_us is not None:
            d["gpu_p50_ms"] = round(float(np.percentile(gpu_us, 50)) / 1e3, 3)
            d["gpu_p99_ms"] = round(float(np.percentile(gpu_us, 99)) / 1e3, 3)
        return d

    def check(out):
        nonlocal ref
        if ref is None:
            ref = out.copy()
        assert np.array_equal(out, ref), "serving results differ between runs"

    def replay(mode, arrival):
        sv = capi.QFMServer(fidx, **modes[mode])
        out = torch.zeros(npat, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        lat = np.zeros(nreq)
        mk = sv.replay(pats, off, first, arrival, out, lat)
        st = sv.stats()
        sv.close()
        check(out)
        return summary(mk, lat, st)

    # the plain path a caller writes without the server: for each request
    # in arrival order, copy its patterns and offsets in, count, copy the
    # counts out, wait; per-request GPU time from CUDA events
    d_pat = torch.empty(int(off[-1]) + 16, dtype=torch.uint8, device="cuda")
    d_off = torch.empty(nreq and int((first[1:] - first[:-1]).max()) + 1, dtype=torch.int64, device="cuda")
    d_out = torch.empty_like(d_off)
    h_off = torch.empty_like(d_off, device="cpu").pin_memory()
    stream = torch.cuda.current_stream()

    def plain_loop(arrival):
        out = torch.zeros(npat, dtype=torch.int64).pin_memory()
        lat = np.zeros(nreq)
        gpu = np.zeros(nreq)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tp = pats_t
        t_start = time.perf_counter()
        for r in range(nreq):
            while time.perf_counter() - t_start < arrival[r]:
                pass
            a, b = int(first[r]), int(first[r + 1])
            pa, pb = int(off[a]), int(off[b])
            h_off[: b - a + 1].copy_(torch.from_numpy((off[a:b + 1] - off[a]).view(np.int64)))
            e0.record(stream)
            d_pat[: pb - pa].copy_(tp[pa:pb], non_blocking=True)
            d_off[: b - a + 1].copy_(h_off[: b - a + 1], non_blocking=True)
            capi.qfm_count(fidx, d_pat, d_off[: b - a + 1], d_out[: b - a])
            out[a:b].copy_(d_out[: b - a], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            lat[r] = (time.perf_counter() - t_start - arrival[r]) * 1e6
            gpu[r] = e0.elapsed_time(e1) * 1e3
        mk = time.perf_counter() - t_start
        check(out.numpy().view(np.uint64))
        return summary(mk, lat, gpu_us=gpu)

    arms = dict(modes)
    arms["plain_qfm_count_loop"] = None
    run = {m: (lambda arr, m=m: plain_loop(arr) if arms[m] is None else replay(m, arr)) for m in arms}
    mean_req = npat / nreq
    # the batching server first: an untimed warm-up replay (after seconds of
    # light GPU load the first replay ran with a p99 of up to ~4 ms), its
    # closed-loop capacity, then Poisson arrivals at 0.5 .. 1.2x of it
    replay("batched", np.zeros(nreq))
    cap = {"batched": replay("batched", np.zeros(nreq))}
    capacity = cap["batched"]["patterns_per_s"]
    for f in (0.5, 0.8, 1.0, 1.2):
        lam = f * capacity / mean_req                                # requests per second
        arrival = np.cumsum(rng.exponential(1.0 / lam, nreq))
        res[f"serving_poisson_{f}x"] = {"batched": replay("batched", arrival)}
        log(f"[bench] serving {f}x batched capacity: batched "
            f"{res[f'serving_poisson_{f}x']['batched']['patterns_per_s'] / 1e6:.1f} M/s p99 "
            f"{res[f'serving_poisson_{f}x']['batched']['p99_ms']} ms")
    # the other arms: closed-loop capacity, then Poisson arrivals at
    # fractions of each arm's own capacity (loads it sustains)
    for m in arms:
        if m != "batched":
            cap[m] = run[m](np.zeros(nreq))
    res["serving_closed_loop"] = cap
    for f in (0.5, 0.8):
        row = {}
        for m in arms:
            if m == "batched":
                continue
            lam = f * cap[m]["patterns_per_s"] / mean_req
            row[m] = run[m](np.cumsum(rng.exponential(1.0 / lam, nreq)))
        res[f"serving_poisson_{f}x_own_capacity"] = row
        log(f"[bench] serving {f}x own capacity: " + ", ".join(
            f"{m} {v['patterns_per_s'] / 1e6:.1f} M/s p99 {v['p99_ms']} ms" for m, v in row.items()))
    fidx.free()
    return res


def parse_cpulist(text: str) -> set:
    """'0-3,8,10-11' -> {0, 1, 2, 3, 8, 10, 11}."""
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        else:
            cpus.add(int(part))
    return cpus


def bind_to_gpu_node(gpu_index: int) -> dict:
    """Run on the host cores local to the GPU (its PCI device's local_cpulist)
    when some of them are allowed, so that pinned host buffers live on the
    GPU's own memory node; reports what was found and done."""
    info = {"gpu_numa_node": None, "bound_cores": None}
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dev = Path("/sys/bus/pci/devices") / ("0000:" + bus.split(":", 1)[1].lower())
        info["gpu_numa_node"] = int((dev / "numa_node").read_text().strip())
        local = parse_cpulist((dev / "local_cpulist").read_text())
        allowed = os.sched_getaffinity(0)
        both = local & allowed
        if both and both != allowed:
            os.sched_setaffinity(0, both)
        info["bound_cores"] = len(both) if both else None
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    return info


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args, n, text, q):
    """The oracle as it stands on a bounded sample, on all host cores: the
    first 2^k queries answered by the threaded sort + sweep (the text cut into
    one chunk per core, each chunk answering its own sorted queries)."""
    import oracle
    cores = host_cores()
    sample = q[: 1 << args.cpu_log_sample].copy()
    oracle.rank(text, n, 2, sample[:1024], 1, threads=cores)      # load the library, touch the text
    t0 = time.perf_counter()
    _, rc = oracle.rank(text, n, 2, sample, 1, threads=cores)
    dt = time.perf_counter() - t0
    assert rc == 0
    return {"value": round(sample.size / dt / 1e9, 6), "unit": "Gqueries/s", "cores": cores, "kind": "oracle",
            "sample": f"first 2^{args.cpu_log_sample} of the queries over the full 2^{args.log_n}-bit text "
                      f"(threaded sort + sweep, one text chunk per core), {dt:.1f}s"}


def cpu_baseline_fm(args, cores=None):
    """QuadFm on the host: the oracle's brute-force counts (direct comparison
    at every text position) of a sample of the count workload's patterns,
    one slice of patterns per core."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_2602_04103_gb300 import workloads
    cores = cores or host_cores()
    text, pats, off = workloads.fm_inputs(args.fm_log_n, args.fm_m)
    k = min(args.cpu_fm_sample, off.size - 1)
    sub_off = off[: k + 1]
    cuts = np.linspace(0, k, cores + 1).astype(np.int64)

    def part(i):
        a, b = int(cuts[i]), int(cuts[i + 1])
        return oracle.count_brute_batch(text, pats[int(sub_off[a]):int(sub_off[b])],
                                        (sub_off[a:b + 1] - sub_off[a]).astype(np.uint64))

    oracle.count_brute_batch(text, pats[:16], np.array([0, 16], dtype=np.uint64))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(part, range(cores)))
    dt = time.perf_counter() - t0
    return {"value": round(k / dt, 1), "unit": "patterns/s", "cores": cores, "kind": "oracle",
            "sample": f"first {k} patterns of the 10^7-pattern workload over the 2^{args.fm_log_n}-char text, "
                      f"brute-force counts, {dt:.1f}s"}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as the reference arm: each step answers a bounded sample
    of the workload's queries over the full text."""
    import oracle
    from paper_2602_04103_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n = 1 << args.log_n
    cores = host_cores()
    text, q = workloads.birank_inputs(args.log_n, args.log_m)
    sample = q[: 1 << args.ref_log_sample].copy()
    for _ in range(args.warmup):
        oracle.rank(text, n, 2, sample[: 1 << 12], 1, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rank(text, n, 2, sample, 1, threads=cores)
    dt = time.perf_counter() - t0
    value = args.steps * sample.size / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gqueries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"BiRank sigma=2 rank(q), n=2^{args.log_n} i.i.d. bits p=0.5, 2^{args.log_m} "
                                   f"uniform uint64 queries per GPU", "n_bits": n, "queries_per_gpu": 1 << args.log_m},
            "cpu_baseline": {"value": round(value, 6), "unit": "Gqueries/s", "cores": cores, "kind": "oracle",
                             "sample": f"2^{args.ref_log_sample} of the queries per step (threaded sort + sweep "
                                       f"over the full text, one text chunk per core)"},
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
    ap.add_argument("--fm-log-n", type=int, default=26)
    ap.add_argument("--fm-m", type=int, default=10_000_000)
    ap.add_argument("--cpu-log-sample", type=int, default=26,
                    help="log2 of the queries the CPU oracle answers for cpu_baseline (all host cores)")
    ap.add_argument("--cpu-fm-sample", type=int, default=2048,
                    help="patterns of the QuadFm CPU baseline (oracle brute-force counts, all host cores)")
    ap.add_argument("--ref-log-sample", type=int, default=25,
                    help="log2 of the queries per step of --impl reference")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--layout", type=int, choices=[0, 1, 2, 3, 4], default=None,
                    help="fixed layout for the headline (skips the tuned build and the probe)")
    ap.add_argument("--tuning", type=int, nargs=3, default=[1, 512, 0], metavar=("K", "THREADS", "LOAD"))
    ap.add_argument("--serve-requests", type=int, default=8000)
    ap.add_argument("--serve-log-n", type=int, default=28)
    ap.add_argument("--serve-stream-calls", action="store_true",
                    help="also run the batching server without CUDA graphs")
    ap.add_argument("--only", choices=["fm", "fm_locate", "fm_approx", "fm_policies", "quadrank", "serving", "probe",
                                       "layouts"],
                    default=None, help="run one extra row alone and print it (profiling runs)")
    args = ap.parse_args()
    if args.only:
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.current_stream()
        if args.only in ("fm", "fm_locate", "fm_approx"):
            res = run_fm(args, stream, part=args.only[3:] or "all")
        elif args.only == "fm_policies":
            res = fm_policies(args, stream)
        elif args.only == "serving":
            res = run_serving(args)
        elif args.only == "layouts":
            res = run_layouts(args, stream)
        elif args.only == "probe":
            res = {"random_32B_requests_G_per_s": round(probe_ceiling(stream), 3),
                   "random_128B_quad_requests_G_per_s": round(probe_ceiling(stream, quad128=True), 3),
                   "probe": "qr_probe_gather: 2^26 random 32-byte loads over a 4 GiB buffer, 4 in flight per "
                            "thread; 2^26 random 128-byte records read quad-cooperatively, 1 or 2 per thread"}
        else:
            res = run_quadrank(args, stream, peaks()[0])
        print(json.dumps(res), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.warmup < 3:
        log("[bench] warmup raised to 3")
        args.warmup = 3
    run_ours(args)


if __name__ == "__main__":
    main()
