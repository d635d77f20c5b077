// C-ABI entry points of the rank side (quadrank.h): argument checks, index
// allocation, launches, the host-buffer pipeline and status handling.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "qr_common.cuh"

namespace qr {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? QR_ENOMEM : QR_ECUDA;
}

const DeviceProps& device_props() {
    static thread_local DeviceProps cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    DeviceProps& p = cache[dev & 63];
    if (p.device != dev) {
        p.device = dev;
        cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&p.l2_bytes, cudaDevAttrL2CacheSize, dev);
        if (p.sms <= 0) p.sms = 1;
    }
    return p;
}

uint64_t block_chars(int sigma, int layout) {
    if (layout == QR_LAYOUT_SECTOR) return sigma == 2 ? kB2s : kB4s;
    if (layout == QR_LAYOUT_LINE128) return sigma == 2 ? kB2L : kB4L;
    if (layout == QR_LAYOUT_INLINE32) return sigma == 2 ? kB2w : kB4w;
    if (layout == QR_LAYOUT_INLINE32X2) return kB2x;
    if (layout == QR_LAYOUT_INLINE24_8) return kB4w;
    return sigma == 2 ? kB2 : kB4;
}
uint64_t super_lines(int sigma, int layout) {
    if (layout == QR_LAYOUT_LINE128) return sigma == 2 ? kSuper2L : kSuper4L;
    if (inline_layout(layout)) return 1ull << l0_shift(layout);
    return sigma == 2 ? kSuper2 : kSuper4;
}
uint64_t line_bytes(int layout) { return layout == QR_LAYOUT_LINE128 ? 128 : 64; }
uint64_t super_entry_bytes(int sigma, int layout) {
    if (inline_layout(layout)) return sigma == 2 ? 8 : 32;
    return sigma == 2 ? 4 : 16;
}

static int tuning_ok(const qr_tuning_t& t) {
    const int k = t.queries_per_thread;
    if (k != 1 && k != 2 && k != 4 && k != 8) return 0;
    if (t.block_threads < 64 || t.block_threads > 512 || (t.block_threads & 31)) return 0;
    if (t.load_mode < 0 || t.load_mode > 4) return 0;
    if (t.grid_blocks < 0) return 0;
    return 1;
}

static void free_index(qr_index* idx) {
    if (!idx) return;
    if (idx->lines) cudaFree(idx->lines);
    if (idx->supers) cudaFree(idx->supers);
    if (idx->status) cudaFree(idx->status);
    if (idx->stage) cudaFree(idx->stage);
    for (auto& s : idx->pipe)
        if (s) cudaStreamDestroy(s);
    for (auto& e : idx->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : idx->region_ev)
        if (e) cudaEventDestroy(e);
    delete idx;
}

}  // namespace qr

using namespace qr;

extern "C" {

const char* qr_last_error(void) { return g_last_error.c_str(); }

int qr_abi_version(void) { return 1; }

int qr_build_ex(const uint64_t* text, uint64_t n, int sigma, int text_on_device, int layout, void* stream,
                qr_index** out) {
    if (!out) return fail(QR_EINVAL, "qr_build: out is NULL");
    *out = nullptr;
    if (sigma != 2 && sigma != 4) return fail(QR_EINVAL, "qr_build: sigma must be 2 or 4");
    if (layout != QR_LAYOUT_PAPER && layout != QR_LAYOUT_SECTOR && layout != QR_LAYOUT_LINE128 &&
        layout != QR_LAYOUT_INLINE32 && layout != QR_LAYOUT_INLINE32X2 && layout != QR_LAYOUT_INLINE24_8)
        return fail(QR_EINVAL, "qr_build: unknown layout");
    if (layout == QR_LAYOUT_INLINE32X2 && sigma != 2)
        return fail(QR_EINVAL, "qr_build: QR_LAYOUT_INLINE32X2 is sigma 2 only");
    if (layout == QR_LAYOUT_INLINE24_8 && sigma != 4)
        return fail(QR_EINVAL, "qr_build: QR_LAYOUT_INLINE24_8 is sigma 4 only");
    if (sigma == 2 && n >= (1ull << 43)) return fail(QR_EINVAL, "qr_build: sigma 2 needs n < 2^43");
    if (sigma == 4 && n >= (1ull << 45)) return fail(QR_EINVAL, "qr_build: sigma 4 needs n < 2^45");
    if (!text && n > 0) return fail(QR_EINVAL, "qr_build: text is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    qr_index* idx = new qr_index();
    cudaGetDevice(&idx->device);
    idx->sigma = sigma;
    idx->layout = layout;
    idx->n = n;
    // default launch tuning per layout (the best measured on GB300; qr_autotune refines it)
    if (layout == QR_LAYOUT_PAPER) idx->tune = qr_tuning_t{4, 512, 4, 0};
    else idx->tune = qr_tuning_t{1, 512, 0, 0};
    const uint64_t B = block_chars(sigma, layout);
    const uint64_t per = super_lines(sigma, layout);
    idx->nblocks = n / B + 1;
    idx->nsuper = (idx->nblocks + per - 1) / per;
    cudaError_t e = cudaMalloc((void**)&idx->lines, line_bytes(layout) * idx->nblocks);
    if (e == cudaSuccess) e = cudaMalloc(&idx->supers, super_entry_bytes(sigma, layout) * idx->nsuper);
    if (e == cudaSuccess) e = cudaMalloc((void**)&idx->status, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(idx->status, 0, 64, s);
    if (e != cudaSuccess) {
        free_index(idx);
        return cuda_fail(e, "qr_build: allocation");
    }
    const uint64_t nwords = sigma == 2 ? (n + 63) / 64 : (n + 31) / 32;
    const uint64_t* d_text = text;
    uint64_t* tmp = nullptr;
    if (!text_on_device && nwords > 0) {
        e = cudaMallocAsync((void**)&tmp, nwords * 8, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, text, nwords * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            if (tmp) cudaFreeAsync(tmp, s);
            cudaStreamSynchronize(s);
            free_index(idx);
            return cuda_fail(e, "qr_build: text upload");
        }
        d_text = tmp;
    }
    int rc = build_rank_index(idx, d_text, s);
    if (tmp) cudaFreeAsync(tmp, s);
    e = cudaStreamSynchronize(s);
    if (rc == QR_OK && e != cudaSuccess) rc = cuda_fail(e, "qr_build: synchronize");
    if (rc != QR_OK) {
        free_index(idx);
        return rc;
    }
    *out = idx;
    return QR_OK;
}

int qr_build(const uint64_t* text, uint64_t n, int sigma, int text_on_device, void* stream, qr_index** out) {
    return qr_build_ex(text, n, sigma, text_on_device, QR_LAYOUT_PAPER, stream, out);
}

static int check_query(const qr_index* idx, const void* q, const void* out, uint64_t m, const char* who) {
    if (!idx) return fail(QR_EINVAL, std::string(who) + ": index is NULL");
    if (m > 0 && (!q || !out)) return fail(QR_EINVAL, std::string(who) + ": NULL buffer");
    return QR_OK;
}

int qr_rank(const qr_index* idx, const uint64_t* q, uint64_t m, int c, uint64_t* out, void* stream) {
    int rc = check_query(idx, q, out, m, "qr_rank");
    if (rc) return rc;
    if (c < 0 || c >= idx->sigma) return fail(QR_EINVAL, "qr_rank: symbol out of range");
    return launch_rank(idx, q, nullptr, c, m, out, 0, (cudaStream_t)stream);
}

int qr_rank_c(const qr_index* idx, const uint64_t* q, const uint8_t* c, uint64_t m, uint64_t* out, void* stream) {
    int rc = check_query(idx, q, out, m, "qr_rank_c");
    if (rc) return rc;
    if (m > 0 && !c) return fail(QR_EINVAL, "qr_rank_c: c is NULL");
    return launch_rank(idx, q, c, 0, m, out, 0, (cudaStream_t)stream);
}

int qr_rank4(const qr_index* idx, const uint64_t* q, uint64_t m, uint64_t* out4, void* stream) {
    int rc = check_query(idx, q, out4, m, "qr_rank4");
    if (rc) return rc;
    if (idx->sigma != 4) return fail(QR_EINVAL, "qr_rank4: needs a sigma 4 index");
    if (((uintptr_t)out4 & 15) != 0) return fail(QR_EINVAL, "qr_rank4: out4 must be 16-byte aligned");
    return launch_rank(idx, q, nullptr, 0, m, out4, 1, (cudaStream_t)stream);
}

int qr_prefix_rank(const qr_index* idx, const uint64_t* q, uint64_t m, int c, uint64_t* out, void* stream) {
    int rc = check_query(idx, q, out, m, "qr_prefix_rank");
    if (rc) return rc;
    if (idx->sigma != 4) return fail(QR_EINVAL, "qr_prefix_rank: needs a sigma 4 index");
    if (c < 0 || c > 3) return fail(QR_EINVAL, "qr_prefix_rank: symbol out of range");
    return launch_rank(idx, q, nullptr, c, m, out, 2, (cudaStream_t)stream);
}

int qr_rank_chain(const qr_index* idx, const uint64_t* q0, uint64_t nchains, uint64_t steps, int c, uint64_t* out2,
                  void* stream) {
    int rc = check_query(idx, q0, out2, nchains, "qr_rank_chain");
    if (rc) return rc;
    if (steps == 0) return fail(QR_EINVAL, "qr_rank_chain: steps must be >= 1");
    if (c < 0 || c >= idx->sigma) return fail(QR_EINVAL, "qr_rank_chain: symbol out of range");
    return launch_chain(idx, q0, nchains, steps, c, out2, (cudaStream_t)stream);
}

// Host-buffer pipeline: chunks go round-robin to kPipe internal streams;
// each chunk is copied in, ranked and copied out on its stream, so the copies
// of some chunks overlap the kernels and copy-outs of others (the copy
// engines of both directions and the SMs work at once).
static int host_pipeline(qr_index* idx, const uint64_t* qh, const uint8_t* ch, uint64_t m, int c, uint64_t* outh,
                         int rank4, cudaStream_t caller) {
    constexpr int P = qr_index::kPipe;
    const uint64_t chunk = 1ull << 23;
    const uint64_t out_per = rank4 ? 32 : 8;
    const size_t slot_bytes = chunk * (8 + 1 + out_per);
    const size_t need = P * slot_bytes;
    if (idx->stage_bytes < need) {
        if (idx->stage) {
            cudaStreamSynchronize(caller);
            for (auto& p : idx->pipe)
                if (p) cudaStreamSynchronize(p);
            cudaFree(idx->stage);
            idx->stage = nullptr;
            idx->stage_bytes = 0;
        }
        QR_CUDA_TRY(cudaMalloc(&idx->stage, need));
        idx->stage_bytes = need;
    }
    for (auto& p : idx->pipe)
        if (!p) QR_CUDA_TRY(cudaStreamCreateWithFlags(&p, cudaStreamNonBlocking));
    for (auto& e : idx->ev)
        if (!e) QR_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    QR_CUDA_TRY(cudaEventRecord(idx->ev[P], caller));
    for (auto& p : idx->pipe) QR_CUDA_TRY(cudaStreamWaitEvent(p, idx->ev[P], 0));
    for (uint64_t off = 0, k = 0; off < m; off += chunk, k++) {
        const uint64_t len = m - off < chunk ? m - off : chunk;
        cudaStream_t st = idx->pipe[k % P];
        char* base = (char*)idx->stage + (k % P) * slot_bytes;
        uint64_t* dq = (uint64_t*)base;
        uint64_t* dout = (uint64_t*)(base + chunk * 8);
        uint8_t* dc = (uint8_t*)(base + chunk * (8 + out_per));
        QR_CUDA_TRY(cudaMemcpyAsync(dq, qh + off, len * 8, cudaMemcpyHostToDevice, st));
        if (ch) QR_CUDA_TRY(cudaMemcpyAsync(dc, ch + off, len, cudaMemcpyHostToDevice, st));
        int rc = launch_rank(idx, dq, ch ? dc : nullptr, c, len, dout, rank4, st);
        if (rc) return rc;
        QR_CUDA_TRY(cudaMemcpyAsync(outh + off * (out_per / 8), dout, len * out_per, cudaMemcpyDeviceToHost, st));
    }
    for (int p = 0; p < P; p++) {
        QR_CUDA_TRY(cudaEventRecord(idx->ev[p], idx->pipe[p]));
        QR_CUDA_TRY(cudaStreamWaitEvent(caller, idx->ev[p], 0));
    }
    QR_CUDA_TRY(cudaStreamSynchronize(caller));
    return QR_OK;
}

int qr_rank_host(qr_index* idx, const uint64_t* q_host, const uint8_t* c_host, uint64_t m, int c,
                 uint64_t* out_host, void* stream) {
    int rc = check_query(idx, q_host, out_host, m, "qr_rank_host");
    if (rc) return rc;
    if (c >= 0 && c >= idx->sigma) return fail(QR_EINVAL, "qr_rank_host: symbol out of range");
    if (c < 0 && m > 0 && !c_host) return fail(QR_EINVAL, "qr_rank_host: c_host is NULL");
    if (m == 0) return QR_OK;
    return host_pipeline(idx, q_host, c < 0 ? c_host : nullptr, m, c < 0 ? 0 : c, out_host, 0,
                         (cudaStream_t)stream);
}

int qr_rank4_host(qr_index* idx, const uint64_t* q_host, uint64_t m, uint64_t* out4_host, void* stream) {
    int rc = check_query(idx, q_host, out4_host, m, "qr_rank4_host");
    if (rc) return rc;
    if (idx->sigma != 4) return fail(QR_EINVAL, "qr_rank4_host: needs a sigma 4 index");
    if (m == 0) return QR_OK;
    return host_pipeline(idx, q_host, nullptr, m, 0, out4_host, 1, (cudaStream_t)stream);
}

int qr_info(const qr_index* idx, qr_info_t* info) {
    if (!idx || !info) return fail(QR_EINVAL, "qr_info: NULL argument");
    info->n = idx->n;
    info->sigma = idx->sigma;
    info->layout = idx->layout;
    info->block_chars = block_chars(idx->sigma, idx->layout);
    info->super_blocks = super_lines(idx->sigma, idx->layout);
    info->line_bytes = line_bytes(idx->layout);
    info->nblocks = idx->nblocks;
    info->nsuper = idx->nsuper;
    info->bytes_blocks = info->line_bytes * idx->nblocks;
    info->bytes_super = super_entry_bytes(idx->sigma, idx->layout) * idx->nsuper;
    return QR_OK;
}

int qr_layout_ptrs(const qr_index* idx, const void** lines, const void** supers) {
    if (!idx) return fail(QR_EINVAL, "qr_layout_ptrs: NULL index");
    if (lines) *lines = idx->lines;
    if (supers) *supers = idx->supers;
    return QR_OK;
}

int qr_copy_layout(const qr_index* idx, void* lines_dst, void* supers_dst, void* stream) {
    if (!idx) return fail(QR_EINVAL, "qr_copy_layout: NULL index");
    cudaStream_t s = (cudaStream_t)stream;
    if (lines_dst)
        QR_CUDA_TRY(cudaMemcpyAsync(lines_dst, idx->lines, line_bytes(idx->layout) * idx->nblocks, cudaMemcpyDefault, s));
    if (supers_dst)
        QR_CUDA_TRY(cudaMemcpyAsync(supers_dst, idx->supers, super_entry_bytes(idx->sigma, idx->layout) * idx->nsuper,
                                    cudaMemcpyDefault, s));
    QR_CUDA_TRY(cudaStreamSynchronize(s));
    return QR_OK;
}

int qr_get_tuning(const qr_index* idx, qr_tuning_t* t) {
    if (!idx || !t) return fail(QR_EINVAL, "qr_get_tuning: NULL argument");
    *t = idx->tune;
    return QR_OK;
}

int qr_set_tuning(qr_index* idx, const qr_tuning_t* t) {
    if (!idx || !t) return fail(QR_EINVAL, "qr_set_tuning: NULL argument");
    if (!tuning_ok(*t)) return fail(QR_EINVAL, "qr_set_tuning: invalid tuning");
    if (idx->layout == QR_LAYOUT_LINE128 && t->queries_per_thread > 2)
        return fail(QR_EINVAL, "qr_set_tuning: the 128-byte line layout takes 1 or 2 queries per thread");
    idx->tune = *t;
    return QR_OK;
}

static int run_mode(qr_index* idx, const uint64_t* q, uint64_t m, int mode, int c, const uint8_t* cv, uint64_t* out,
                    cudaStream_t s) {
    if (mode == 0) return launch_rank(idx, q, nullptr, c, m, out, 0, s);
    if (mode == 1) return launch_rank(idx, q, cv, 0, m, out, 0, s);
    return launch_rank(idx, q, nullptr, 0, m, out, 1, s);
}

int qr_autotune(qr_index* idx, const uint64_t* q, uint64_t m, int mode, int c, const uint8_t* c_vec, uint64_t* out,
                void* stream, qr_tuning_t* best) {
    if (!idx || !q || !out || m == 0) return fail(QR_EINVAL, "qr_autotune: NULL argument or m = 0");
    if (mode < 0 || mode > 2) return fail(QR_EINVAL, "qr_autotune: mode must be 0, 1 or 2");
    if (mode == 0 && (c < 0 || c >= idx->sigma)) return fail(QR_EINVAL, "qr_autotune: symbol out of range");
    if (mode == 1 && !c_vec) return fail(QR_EINVAL, "qr_autotune: c_vec is NULL");
    if (mode == 2 && idx->sigma != 4) return fail(QR_EINVAL, "qr_autotune: rank4 needs sigma 4");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    QR_CUDA_TRY(cudaEventCreate(&e0));
    QR_CUDA_TRY(cudaEventCreate(&e1));
    const qr_tuning_t saved = idx->tune;
    qr_tuning_t win = saved;
    // the candidates tune the direct kernels, so time those alone
    const int saved_mode = idx->batch_mode;
    idx->batch_mode = QR_BATCH_DIRECT;
    float win_ms = 1e30f;
    const int ks[] = {1, 2, 4, 8}, ths[] = {128, 256, 512};
    const int nload = idx->layout == QR_LAYOUT_PAPER ? 5 : 1;
    int rc = QR_OK;
    for (int li = 0; li < nload && rc == QR_OK; li++)
        for (int k : ks)
            for (int th : ths) {
                if (idx->layout == QR_LAYOUT_LINE128 && k > 2) continue;  // 1 or 2 lines per lane
                idx->tune = qr_tuning_t{k, th, li, 0};
                rc = run_mode(idx, q, m, mode, c, c_vec, out, s);  // warm-up
                float bestk = 1e30f;
                for (int r = 0; r < 3 && rc == QR_OK; r++) {
                    cudaEventRecord(e0, s);
                    rc = run_mode(idx, q, m, mode, c, c_vec, out, s);
                    cudaEventRecord(e1, s);
                    cudaError_t e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) rc = cuda_fail(e, "qr_autotune: timing");
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < bestk) bestk = ms;
                }
                if (rc != QR_OK) break;
                if (bestk < win_ms) {
                    win_ms = bestk;
                    win = idx->tune;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    idx->batch_mode = saved_mode;
    idx->tune = rc == QR_OK ? win : saved;
    if (best) *best = idx->tune;
    return rc;
}

static constexpr uint64_t kTuneSample = 1ull << 24;  // queries timed per autotuning candidate

static double layout_overhead(int sigma, int layout, uint64_t n) {
    const uint64_t B = block_chars(sigma, layout), per = super_lines(sigma, layout);
    const uint64_t nb = n / B + 1, ns = (nb + per - 1) / per;
    const double bytes = (double)line_bytes(layout) * nb + (double)super_entry_bytes(sigma, layout) * ns;
    const double text = sigma == 2 ? n / 8.0 : n / 4.0;
    return n ? bytes / text - 1.0 : 0.0;
}

int qr_build_tuned(const uint64_t* text, uint64_t n, int sigma, int text_on_device, double max_overhead,
                   const uint64_t* q, uint64_t m, int mode, int c, const uint8_t* c_vec, uint64_t* out, void* stream,
                   qr_index** idx_out, int* layout_out) {
    if (!idx_out) return fail(QR_EINVAL, "qr_build_tuned: idx_out is NULL");
    *idx_out = nullptr;
    qr_index* best = nullptr;
    int best_layout = -1;
    float best_ms = 1e30f;
    cudaStream_t s = (cudaStream_t)stream;
    for (int layout : {QR_LAYOUT_PAPER, QR_LAYOUT_SECTOR, QR_LAYOUT_LINE128, QR_LAYOUT_INLINE32,
                       QR_LAYOUT_INLINE32X2, QR_LAYOUT_INLINE24_8}) {
        if (layout == QR_LAYOUT_INLINE32X2 && sigma != 2) continue;
        if (layout == QR_LAYOUT_INLINE24_8 && sigma != 4) continue;
        if (sigma == 2 || sigma == 4) {
            if (layout_overhead(sigma, layout, n < 4096 ? 1u << 30 : n) > max_overhead) continue;
        }
        qr_index* idx = nullptr;
        int rc = qr_build_ex(text, n, sigma, text_on_device, layout, stream, &idx);
        if (rc != QR_OK) {
            if (best) qr_free(best);
            return rc;
        }
        // the direct kernels are tuned on a prefix of the batch; the layouts are
        // then compared on the whole batch, by the path the handle takes for it
        qr_tuning_t t;
        rc = qr_autotune(idx, q, m < kTuneSample ? m : kTuneSample, mode, c, c_vec, out, stream, &t);
        if (rc != QR_OK) {
            qr_free(idx);
            if (best) qr_free(best);
            return rc;
        }
        // time the tuned kernel once more for the comparison across layouts
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float ms = 1e30f;
        for (int r = 0; r < 3; r++) {
            cudaEventRecord(e0, s);
            rc = run_mode(idx, q, m, mode, c, c_vec, out, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float x = 0;
            cudaEventElapsedTime(&x, e0, e1);
            if (x < ms) ms = x;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (ms < best_ms) {
            if (best) qr_free(best);
            best = idx;
            best_ms = ms;
            best_layout = layout;
        } else {
            qr_free(idx);
        }
    }
    if (!best) return fail(QR_EINVAL, "qr_build_tuned: no layout within max_overhead");
    *idx_out = best;
    if (layout_out) *layout_out = best_layout;
    return QR_OK;
}

int qr_set_batch_mode(qr_index* idx, int mode) {
    if (!idx) return fail(QR_EINVAL, "qr_set_batch_mode: NULL index");
    if (mode != QR_BATCH_AUTO && mode != QR_BATCH_DIRECT && mode != QR_BATCH_REGIONS)
        return fail(QR_EINVAL, "qr_set_batch_mode: unknown mode");
    idx->batch_mode = mode;
    return QR_OK;
}

int qr_rank_plan(const qr_index* idx, uint64_t m, int rank4, int* plan) {
    if (!idx || !plan) return fail(QR_EINVAL, "qr_rank_plan: NULL argument");
    if (rank4 < 0 || rank4 > 2) return fail(QR_EINVAL, "qr_rank_plan: rank4 must be 0, 1 or 2");
    bool regions = false;
    if (m > 0 && region_supported(idx, rank4) && idx->batch_mode != QR_BATCH_DIRECT)
        regions = idx->batch_mode == QR_BATCH_REGIONS ? m < (1ull << 32) : region_auto(idx, m);
    *plan = regions ? QR_BATCH_REGIONS : QR_BATCH_DIRECT;
    return QR_OK;
}

int qr_region_timing(qr_index* idx, int enable, float* ms3) {
    if (!idx) return fail(QR_EINVAL, "qr_region_timing: NULL index");
    if (ms3) {
        if (!idx->region_ev[3]) return fail(QR_EINVAL, "qr_region_timing: timing was never enabled");
        QR_CUDA_TRY(cudaEventSynchronize(idx->region_ev[3]));
        for (int k = 0; k < 3; k++) {
            float x = 0;
            QR_CUDA_TRY(cudaEventElapsedTime(&x, idx->region_ev[k], idx->region_ev[k + 1]));
            ms3[k] = x;
        }
    }
    if (enable)
        for (auto& e : idx->region_ev)
            if (!e) QR_CUDA_TRY(cudaEventCreate(&e));
    idx->region_timing = enable != 0;
    return QR_OK;
}

int qr_set_region_tuning(qr_index* idx, int variant) {
    if (!idx) return fail(QR_EINVAL, "qr_set_region_tuning: NULL index");
    if (variant < 0 || variant > 3) return fail(QR_EINVAL, "qr_set_region_tuning: variant must be 0..3");
    idx->region_variant = variant;
    return QR_OK;
}

int qr_set_region_fault(qr_index* idx, int withhold) {
    if (!idx) return fail(QR_EINVAL, "qr_set_region_fault: NULL index");
    idx->region_withhold = withhold != 0;
    return QR_OK;
}

int qr_release_scratch(void) { return region_trim(); }

int qr_status(qr_index* idx, void* stream) {
    if (!idx) return fail(QR_EINVAL, "qr_status: NULL index");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t v = 0;
    QR_CUDA_TRY(cudaMemcpyAsync(&v, idx->status, 4, cudaMemcpyDeviceToHost, s));
    QR_CUDA_TRY(cudaMemsetAsync(idx->status, 0, 4, s));
    QR_CUDA_TRY(cudaStreamSynchronize(s));
    return (int)v;
}

int qr_free(qr_index* idx) {
    if (!idx) return QR_OK;
    cudaDeviceSynchronize();
    free_index(idx);
    return QR_OK;
}

int qr_probe_gather(const void* buf, uint64_t nrec, int bytes, int load_bytes, uint64_t m, uint64_t seed,
                    uint64_t* out, int queries_per_thread, int block_threads, void* stream) {
    if (bytes != 16 && bytes != 32 && bytes != 64 && bytes != 128) return fail(QR_EINVAL, "probe: bytes");
    if (load_bytes != 16 && load_bytes != 32 && !(load_bytes == 128 && bytes == 128))
        return fail(QR_EINVAL, "probe: load_bytes");
    if (nrec == 0 || !buf || (m > 0 && !out)) return fail(QR_EINVAL, "probe: empty buffer");
    if (((uintptr_t)buf & 15) != 0) return fail(QR_EINVAL, "probe: buf must be 16-byte aligned");
    if (block_threads < 64 || block_threads > 1024 || (block_threads & 31)) return fail(QR_EINVAL, "probe: threads");
    return launch_probe(buf, nrec, bytes, load_bytes, m, seed, out, queries_per_thread, block_threads,
                        (cudaStream_t)stream);
}

int qr_probe_l2(const void* buf, uint64_t nrec, int mode, uint64_t nthreads, uint32_t rounds, uint64_t seed,
                uint64_t* out, int block_threads, void* stream) {
    if (mode != 0 && mode != 1) return fail(QR_EINVAL, "qr_probe_l2: mode must be 0 or 1");
    if (nrec == 0 || !buf || (nthreads > 0 && !out)) return fail(QR_EINVAL, "qr_probe_l2: empty buffer");
    if (nrec > (1ull << 40)) return fail(QR_EINVAL, "qr_probe_l2: nrec above 2^40");
    if (((uintptr_t)buf & 31) != 0) return fail(QR_EINVAL, "qr_probe_l2: buf must be 32-byte aligned");
    if (rounds == 0) return fail(QR_EINVAL, "qr_probe_l2: rounds must be >= 1");
    if (block_threads < 64 || block_threads > 256 || (block_threads & 31))
        return fail(QR_EINVAL, "qr_probe_l2: block_threads must be 64..256, a multiple of 32");
    return launch_probe_l2(buf, nrec, mode, nthreads, rounds, seed, out, block_threads, (cudaStream_t)stream);
}

}  // extern "C"
