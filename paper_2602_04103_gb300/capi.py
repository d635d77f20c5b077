"""ctypes binding of libquadrank.so (include/quadrank.h), same entry-point names.

Argument marshalling only: every step of the query path runs in the CUDA
kernels of the library.  Device buffers are torch CUDA tensors (any 8-byte
integer dtype for uint64 data, uint8 for symbols / patterns); host buffers
are numpy arrays or CPU tensors (pinned for full copy bandwidth).  Importing
this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

_SO = Path(__file__).resolve().parent / "_lib" / "libquadrank.so"
if not _SO.exists():
    raise ImportError(f"{_SO} is missing: build it with __graft_entry__.build() "
                      "(nvcc, sm_103a); there is no fallback path")
lib = C.CDLL(str(_SO))

QR_OK, QR_EINVAL, QR_ENOMEM, QR_ECUDA = 0, 1, 2, 3
QR_ERANGE, QR_EBADSYM, QR_ETIMEOUT = 4, 8, 16
QR_LAYOUT_PAPER, QR_LAYOUT_SECTOR, QR_LAYOUT_LINE128 = 0, 1, 2
QR_LAYOUT_INLINE32, QR_LAYOUT_INLINE32X2, QR_LAYOUT_INLINE24_8 = 3, 4, 5
QFM_KEEP_SA = 1
QFM_BOTH_STRANDS = 2

u64, i32, vp = C.c_uint64, C.c_int, C.c_void_p


class qr_info_t(C.Structure):
    _fields_ = [("n", u64), ("sigma", C.c_int32), ("layout", C.c_int32), ("block_chars", u64),
                ("super_blocks", u64), ("line_bytes", u64), ("nblocks", u64), ("nsuper", u64),
                ("bytes_blocks", u64), ("bytes_super", u64)]


class qr_tuning_t(C.Structure):
    _fields_ = [("queries_per_thread", C.c_int32), ("block_threads", C.c_int32), ("load_mode", C.c_int32),
                ("grid_blocks", C.c_int32)]


class QRError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib.qr_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with code {code}: {msg}")
        self.code = code


def _sig(name, args, res=i32):
    f = getattr(lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("qr_last_error", [], C.c_char_p)
_sig("qr_abi_version", [])
_sig("qr_build", [vp, u64, i32, i32, vp, C.POINTER(vp)])
_sig("qr_build_ex", [vp, u64, i32, i32, i32, vp, C.POINTER(vp)])
_sig("qr_rank", [vp, vp, u64, i32, vp, vp])
_sig("qr_rank_c", [vp, vp, vp, u64, vp, vp])
_sig("qr_rank4", [vp, vp, u64, vp, vp])
_sig("qr_prefix_rank", [vp, vp, u64, i32, vp, vp])
_sig("qr_rank_chain", [vp, vp, u64, u64, i32, vp, vp])
_sig("qr_rank_host", [vp, vp, vp, u64, i32, vp, vp])
_sig("qr_rank4_host", [vp, vp, u64, vp, vp])
_sig("qr_info", [vp, C.POINTER(qr_info_t)])
_sig("qr_layout_ptrs", [vp, C.POINTER(vp), C.POINTER(vp)])
_sig("qr_copy_layout", [vp, vp, vp, vp])
_sig("qr_get_tuning", [vp, C.POINTER(qr_tuning_t)])
_sig("qr_set_tuning", [vp, C.POINTER(qr_tuning_t)])
_sig("qr_autotune", [vp, vp, u64, i32, i32, vp, vp, vp, C.POINTER(qr_tuning_t)])
_sig("qr_build_tuned", [vp, u64, i32, i32, C.c_double, vp, u64, i32, i32, vp, vp, vp, C.POINTER(vp),
                        C.POINTER(C.c_int)])
_sig("qr_status", [vp, vp])
_sig("qr_free", [vp])
_sig("qr_probe_gather", [vp, u64, i32, i32, u64, u64, vp, i32, i32, vp])
_sig("qr_probe_l2", [vp, u64, i32, u64, C.c_uint32, u64, vp, i32, vp])
_sig("qr_set_batch_mode", [vp, i32])
_sig("qr_rank_plan", [vp, u64, i32, C.POINTER(C.c_int)])
_sig("qr_region_timing", [vp, i32, C.POINTER(C.c_float)])
_sig("qr_release_scratch", [])
_sig("qr_set_region_tuning", [vp, i32])
_sig("qr_set_region_fault", [vp, i32])


def _check(rc: int, where: str) -> None:
    if rc != QR_OK:
        raise QRError(rc, where)


def ptr(x) -> int | None:
    """Address of a torch tensor / numpy array (None for None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def stream_ptr(stream=None) -> int | None:
    """cudaStream_t of a torch stream (default: torch's current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def numel(x) -> int:
    return x.numel() if hasattr(x, "numel") else x.size


class _Handle:
    """Owner of an opaque library handle (freed by `free`)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return vp(self.handle)


class QRIndex(_Handle):
    """Owner of a qr_index* (freed with qr_free).  The methods allocate the
    output on the queries' device when `out` is None and call the entry point
    of the same name; like those, they are asynchronous on `stream`."""

    def free(self) -> None:
        if self.handle:
            lib.qr_free(self.handle)
            self.handle = None

    def rank(self, q, c, out=None, stream=None):
        """rank(q, c) of every position in q: qr_rank for an int symbol,
        qr_rank_c for a per-query uint8 symbol tensor."""
        import torch
        out = torch.empty_like(q) if out is None else out
        if isinstance(c, int):
            qr_rank(self, q, c, out, stream)
        else:
            qr_rank_c(self, q, c, out, stream)
        return out

    def rank4(self, q, out4=None, stream=None):
        """All four symbol ranks of every position (sigma = 4): an m x 4 tensor."""
        import torch
        out4 = torch.empty((numel(q), 4), dtype=q.dtype, device=q.device) if out4 is None else out4
        qr_rank4(self, q, out4, stream)
        return out4

    def prefix_rank(self, q, c: int, out=None, stream=None):
        """The number of symbols <= c before each position (sigma = 4)."""
        import torch
        out = torch.empty_like(q) if out is None else out
        qr_prefix_rank(self, q, c, out, stream)
        return out

    def status(self, stream=None) -> int:
        return qr_status(self, stream)


def qr_build(text, n: int, sigma: int, stream=None, layout: int = QR_LAYOUT_PAPER) -> QRIndex:
    on_dev = int(hasattr(text, "is_cuda") and text.is_cuda)
    h = vp()
    _check(lib.qr_build_ex(ptr(text), n, sigma, on_dev, layout, stream_ptr(stream), C.byref(h)), "qr_build")
    return QRIndex(h.value)


def qr_rank(idx: QRIndex, q, c: int, out, stream=None) -> None:
    _check(lib.qr_rank(idx, ptr(q), numel(q), c, ptr(out), stream_ptr(stream)), "qr_rank")


def qr_rank_c(idx: QRIndex, q, c, out, stream=None) -> None:
    _check(lib.qr_rank_c(idx, ptr(q), ptr(c), numel(q), ptr(out), stream_ptr(stream)), "qr_rank_c")


def qr_rank4(idx: QRIndex, q, out4, stream=None) -> None:
    _check(lib.qr_rank4(idx, ptr(q), numel(q), ptr(out4), stream_ptr(stream)), "qr_rank4")


def qr_prefix_rank(idx: QRIndex, q, c: int, out, stream=None) -> None:
    _check(lib.qr_prefix_rank(idx, ptr(q), numel(q), c, ptr(out), stream_ptr(stream)), "qr_prefix_rank")


def qr_rank_chain(idx: QRIndex, q0, steps: int, c: int, out2, stream=None) -> None:
    """Dependent query chains (out2: 2 x chains: last position, last rank)."""
    _check(lib.qr_rank_chain(idx, ptr(q0), numel(q0), steps, c, ptr(out2), stream_ptr(stream)), "qr_rank_chain")


def qr_rank_host(idx: QRIndex, q_host, c, out_host, stream=None) -> None:
    """c: an int symbol, or a host uint8 array of per-query symbols."""
    if isinstance(c, int):
        rc = lib.qr_rank_host(idx, ptr(q_host), None, numel(q_host), c, ptr(out_host), stream_ptr(stream))
    else:
        rc = lib.qr_rank_host(idx, ptr(q_host), ptr(c), numel(q_host), -1, ptr(out_host), stream_ptr(stream))
    _check(rc, "qr_rank_host")


def qr_rank4_host(idx: QRIndex, q_host, out4_host, stream=None) -> None:
    _check(lib.qr_rank4_host(idx, ptr(q_host), numel(q_host), ptr(out4_host), stream_ptr(stream)), "qr_rank4_host")


def qr_info(idx: QRIndex) -> dict:
    info = qr_info_t()
    _check(lib.qr_info(idx, C.byref(info)), "qr_info")
    return {k: getattr(info, k) for k, _ in qr_info_t._fields_}


def qr_layout_ptrs(idx: QRIndex) -> tuple[int, int]:
    a, b = vp(), vp()
    _check(lib.qr_layout_ptrs(idx, C.byref(a), C.byref(b)), "qr_layout_ptrs")
    return a.value, b.value


def qr_copy_layout(idx: QRIndex, lines_dst=None, supers_dst=None, stream=None) -> None:
    _check(lib.qr_copy_layout(idx, ptr(lines_dst), ptr(supers_dst), stream_ptr(stream)), "qr_copy_layout")


def qr_get_tuning(idx: QRIndex) -> dict:
    t = qr_tuning_t()
    _check(lib.qr_get_tuning(idx, C.byref(t)), "qr_get_tuning")
    return {k: getattr(t, k) for k, _ in qr_tuning_t._fields_}


def qr_set_tuning(idx: QRIndex, queries_per_thread=4, block_threads=256, load_mode=0, grid_blocks=0) -> None:
    t = qr_tuning_t(queries_per_thread, block_threads, load_mode, grid_blocks)
    _check(lib.qr_set_tuning(idx, C.byref(t)), "qr_set_tuning")


def _mode_args(c, rank4):
    if rank4:
        return 2, 0, None
    if isinstance(c, (int,)):
        return 0, c, None
    return 1, 0, ptr(c)


def qr_autotune(idx: QRIndex, q, out, c=1, rank4=False, stream=None) -> dict:
    """Pick the fastest tuning on these queries (out: device scratch of m, or 4m for rank4)."""
    mode, ci, cv = _mode_args(c, rank4)
    t = qr_tuning_t()
    _check(lib.qr_autotune(idx, ptr(q), numel(q), mode, ci, cv, ptr(out), stream_ptr(stream), C.byref(t)),
           "qr_autotune")
    return {k: getattr(t, k) for k, _ in qr_tuning_t._fields_}


def qr_build_tuned(text, n: int, sigma: int, q, out, c=1, rank4=False, max_overhead=1.0,
                   stream=None) -> tuple[QRIndex, int]:
    """Build every layout within max_overhead, autotune each, return (fastest index, its layout)."""
    mode, ci, cv = _mode_args(c, rank4)
    on_dev = int(hasattr(text, "is_cuda") and text.is_cuda)
    h, lay = vp(), C.c_int()
    _check(lib.qr_build_tuned(ptr(text), n, sigma, on_dev, max_overhead, ptr(q), numel(q), mode, ci, cv, ptr(out),
                              stream_ptr(stream), C.byref(h), C.byref(lay)), "qr_build_tuned")
    return QRIndex(h.value), lay.value


QR_BATCH_AUTO, QR_BATCH_DIRECT, QR_BATCH_REGIONS = 0, 1, 2


def qr_set_batch_mode(idx: QRIndex, mode: int) -> None:
    _check(lib.qr_set_batch_mode(idx, mode), "qr_set_batch_mode")


def qr_rank_plan(idx: QRIndex, m: int, rank4: int = 0) -> int:
    plan = C.c_int()
    _check(lib.qr_rank_plan(idx, m, rank4, C.byref(plan)), "qr_rank_plan")
    return plan.value


def qr_region_timing(idx: QRIndex, enable: bool, read: bool = False) -> list[float] | None:
    """Switch per-pass timing of region-batched calls; with read=True first return the
    last such call's three pass times (sort, rank, unsort) in ms."""
    ms = (C.c_float * 3)()
    _check(lib.qr_region_timing(idx, int(enable), ms if read else None), "qr_region_timing")
    return list(ms) if read else None


def qr_set_region_tuning(idx: QRIndex, variant: int = 0) -> None:
    _check(lib.qr_set_region_tuning(idx, variant), "qr_set_region_tuning")


def qr_set_region_fault(idx: QRIndex, withhold: bool) -> None:
    _check(lib.qr_set_region_fault(idx, int(withhold)), "qr_set_region_fault")


def qr_release_scratch() -> None:
    _check(lib.qr_release_scratch(), "qr_release_scratch")


def qr_status(idx: QRIndex, stream=None) -> int:
    rc = lib.qr_status(idx, stream_ptr(stream))
    if rc in (QR_EINVAL, QR_ECUDA, QR_ENOMEM):
        raise QRError(rc, "qr_status")
    return rc


def qr_probe_gather(buf, nrec: int, nbytes: int, m: int, seed: int, out, queries_per_thread=4,
                    block_threads=256, load_bytes=16, stream=None) -> None:
    _check(lib.qr_probe_gather(ptr(buf), nrec, nbytes, load_bytes, m, seed, ptr(out), queries_per_thread,
                               block_threads, stream_ptr(stream)), "qr_probe_gather")


def qr_probe_l2(buf, nrec: int, mode: int, nthreads: int, rounds: int, seed: int, out, block_threads=256,
                stream=None) -> None:
    """Random 64-byte record reads from an L2-resident buffer (mode 0:
    independent, 4 per thread and round; mode 1: dependent pairs)."""
    _check(lib.qr_probe_l2(ptr(buf), nrec, mode, nthreads, rounds, seed, ptr(out), block_threads,
                           stream_ptr(stream)), "qr_probe_l2")


# ---------------------------------------------------------------- QuadFm (include/quadfm.h)
class qfm_info_t(C.Structure):
    _fields_ = [("n", u64), ("dollar_row", u64), ("C", u64 * 5), ("bytes_rank", u64), ("bytes_table", u64),
                ("kmer", C.c_int32), ("has_sa", C.c_int32), ("sa_sample", C.c_int32), ("reserved", C.c_int32),
                ("bytes_locate", u64)]


_sig("qfm_build", [vp, u64, i32, i32, vp, C.POINTER(vp)])
_sig("qfm_build_ex", [vp, u64, i32, i32, C.c_uint32, vp, C.POINTER(vp)])
_sig("qfm_locate", [vp, vp, vp, u64, vp, vp, u64, C.POINTER(u64), vp])
_sig("qfm_count_approx", [vp, vp, vp, u64, i32, vp, vp])
_sig("qfm_count", [vp, vp, vp, u64, vp, vp])
_sig("qfm_count_ex", [vp, vp, vp, u64, vp, i32, vp])
_sig("qfm_count_stepwise", [vp, vp, vp, u64, vp, vp])
_sig("qfm_count_noalloc", [vp, vp, vp, u64, vp, vp])
_sig("qfm_set_policy", [vp, i32])
_sig("qfm_info", [vp, C.POINTER(qfm_info_t)])
_sig("qfm_export", [vp, vp, vp, vp, vp])
_sig("qfm_rank_index", [vp], vp)
_sig("qfm_status", [vp, vp])
_sig("qfm_free", [vp])


class QFMIndex(_Handle):
    """Owner of a qfm_index* (freed with qfm_free); `count` allocates the
    output when `out` is None and calls qfm_count_ex."""

    def free(self) -> None:
        if self.handle:
            lib.qfm_free(self.handle)
            self.handle = None

    def count(self, patterns, offsets, flags: int = 0, out=None, stream=None):
        """Occurrence counts of the m patterns (2m with QFM_BOTH_STRANDS)."""
        import torch
        m = numel(offsets) - 1
        if out is None:
            n_out = 2 * m if flags & QFM_BOTH_STRANDS else m
            out = torch.empty(n_out, dtype=torch.int64, device=offsets.device)
        qfm_count_ex(self, patterns, offsets, out, flags, stream)
        return out

    def status(self, stream=None) -> int:
        return qfm_status(self, stream)


def qfm_build(codes, n: int | None = None, flags: int = 0, stream=None, sa_sample: int = 0) -> QFMIndex:
    on_dev = int(hasattr(codes, "is_cuda") and codes.is_cuda)
    n = numel(codes) if n is None else n
    h = vp()
    _check(lib.qfm_build_ex(ptr(codes), n, on_dev, flags, sa_sample, stream_ptr(stream), C.byref(h)), "qfm_build")
    return QFMIndex(h.value)


def qfm_count_approx(idx: QFMIndex, patterns, offsets, k: int, out, stream=None) -> None:
    """out[j] = occurrences of pattern j with at most k substitutions (k <= 3)."""
    m = numel(offsets) - 1
    _check(lib.qfm_count_approx(idx, ptr(patterns), ptr(offsets), m, k, ptr(out), stream_ptr(stream)),
           "qfm_count_approx")


def qfm_locate(idx: QFMIndex, patterns, offsets, occ, positions=None, stream=None) -> int:
    """occ (m + 1 device uint64) and, with `positions`, every occurrence's text
    position; returns the total.  QRError with code QR_ERANGE when `positions`
    is too small (occ is valid then)."""
    m = numel(offsets) - 1
    total = u64(0)
    cap = numel(positions) if positions is not None else 0
    _check(lib.qfm_locate(idx, ptr(patterns), ptr(offsets), m, ptr(occ), ptr(positions), cap, C.byref(total),
                          stream_ptr(stream)), "qfm_locate")
    return int(total.value)


def qfm_count(idx: QFMIndex, patterns, offsets, out, stream=None) -> None:
    m = numel(offsets) - 1
    _check(lib.qfm_count(idx, ptr(patterns), ptr(offsets), m, ptr(out), stream_ptr(stream)), "qfm_count")


def qfm_count_ex(idx: QFMIndex, patterns, offsets, out, flags: int = 0, stream=None) -> None:
    """flags = QFM_BOTH_STRANDS: out holds 2m counts (forward, then reverse complements)."""
    m = numel(offsets) - 1
    _check(lib.qfm_count_ex(idx, ptr(patterns), ptr(offsets), m, ptr(out), flags, stream_ptr(stream)),
           "qfm_count_ex")


def qfm_count_stepwise(idx: QFMIndex, patterns, offsets, out, stream=None) -> None:
    m = numel(offsets) - 1
    _check(lib.qfm_count_stepwise(idx, ptr(patterns), ptr(offsets), m, ptr(out), stream_ptr(stream)),
           "qfm_count_stepwise")


def qfm_count_noalloc(idx: QFMIndex, patterns, offsets, out, stream=None) -> None:
    """qfm_count without any device allocation (static scratch; see quadfm.h)."""
    m = numel(offsets) - 1
    _check(lib.qfm_count_noalloc(idx, ptr(patterns), ptr(offsets), m, ptr(out), stream_ptr(stream)),
           "qfm_count_noalloc")


def qfm_set_policy(idx: QFMIndex, policy: int) -> None:
    _check(lib.qfm_set_policy(idx, policy), "qfm_set_policy")


def qfm_info(idx: QFMIndex) -> dict:
    info = qfm_info_t()
    _check(lib.qfm_info(idx, C.byref(info)), "qfm_info")
    d = {k: getattr(info, k) for k, _ in qfm_info_t._fields_}
    d["C"] = list(info.C)
    return d


def qfm_export(idx: QFMIndex, sa=None, bwt=None, table=None, stream=None) -> None:
    _check(lib.qfm_export(idx, ptr(sa), ptr(bwt), ptr(table), stream_ptr(stream)), "qfm_export")


def qfm_status(idx: QFMIndex, stream=None) -> int:
    rc = lib.qfm_status(idx, stream_ptr(stream))
    if rc in (QR_EINVAL, QR_ECUDA, QR_ENOMEM):
        raise QRError(rc, "qfm_status")
    return rc


# ---------------------------------------------------------------- serving
class qfm_server_opts_t(C.Structure):
    _fields_ = [("budget_bytes", u64), ("slots", C.c_int32), ("max_requests_per_batch", C.c_int32),
                ("max_batch_patterns", u64), ("max_batch_bytes", u64), ("poll_us", C.c_int32),
                ("fail_after_batches", C.c_int32), ("use_graph", C.c_int32), ("reserved", C.c_int32)]


class qfm_server_stats_t(C.Structure):
    _fields_ = [("submitted", u64), ("completed", u64), ("pending", u64), ("in_flight", u64), ("batches", u64),
                ("mean_requests_per_batch", C.c_double), ("error", C.c_int32), ("reserved", C.c_int32),
                ("graph_batches", u64)]


_sig("qfm_server_default_opts", [C.POINTER(qfm_server_opts_t)])
_sig("qfm_server_create", [vp, C.POINTER(qfm_server_opts_t), C.POINTER(vp)])
_sig("qfm_server_submit", [vp, vp, vp, u64, vp, C.POINTER(u64)])
_sig("qfm_server_poll", [vp, vp, vp, vp, u64, C.POINTER(u64)])
_sig("qfm_server_drain", [vp, C.c_double])
_sig("qfm_server_stats", [vp, C.POINTER(qfm_server_stats_t)])
_sig("qfm_server_destroy", [vp])
_sig("qfm_server_replay", [vp, vp, vp, vp, u64, vp, vp, vp, C.POINTER(C.c_double)])


class QFMServer:
    """Owner of a qfm_server* (stopped and freed with qfm_server_destroy)."""

    def __init__(self, idx: QFMIndex, **opts):
        o = qfm_server_opts_t()
        _check(lib.qfm_server_default_opts(C.byref(o)), "qfm_server_default_opts")
        for k, v in opts.items():
            setattr(o, k, v)
        h = vp()
        _check(lib.qfm_server_create(idx, C.byref(o), C.byref(h)), "qfm_server_create")
        self.handle, self.idx = h.value, idx

    @property
    def _as_parameter_(self):
        return vp(self.handle)

    def submit(self, patterns, offsets, out) -> int:
        rid = u64()
        _check(lib.qfm_server_submit(self, ptr(patterns), ptr(offsets), numel(offsets) - 1, ptr(out), C.byref(rid)),
               "qfm_server_submit")
        return rid.value

    def poll(self, cap: int = 4096):
        import numpy as np
        ids = np.empty(cap, np.uint64)
        lat = np.empty(cap, np.float64)
        st = np.empty(cap, np.int32)
        n = u64()
        _check(lib.qfm_server_poll(self, ptr(ids), ptr(lat), ptr(st), cap, C.byref(n)), "qfm_server_poll")
        k = n.value
        return ids[:k], lat[:k], st[:k]

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(lib.qfm_server_drain(self, timeout_s), "qfm_server_drain")

    def stats(self) -> dict:
        st = qfm_server_stats_t()
        _check(lib.qfm_server_stats(self, C.byref(st)), "qfm_server_stats")
        return {k: getattr(st, k) for k, _ in qfm_server_stats_t._fields_}

    def replay(self, patterns, offsets, req_first, arrival_s, out, latency_us) -> float:
        mk = C.c_double()
        _check(lib.qfm_server_replay(self, ptr(patterns), ptr(offsets), ptr(req_first), numel(req_first) - 1,
                                     ptr(arrival_s), ptr(out), ptr(latency_us), C.byref(mk)), "qfm_server_replay")
        return mk.value

    def close(self) -> None:
        if self.handle:
            lib.qfm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
