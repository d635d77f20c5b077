// Continuous-batching server for QuadFm counts (host runtime around the
// persistent count kernel).
//
// A worker thread owns `slots` batch slots.  Each slot holds device buffers
// for patterns / offsets / counts carved from the server's device-memory
// budget, pinned host staging of the same sizes, a stream and an event.
// Whenever a slot is free and requests are pending, the worker packs pending
// requests in arrival order into the slot while they fit (pattern bytes,
// pattern count, requests per batch), copies them in, launches the count
// kernel on the slot's stream and copies the counts back.  Requests that
// arrive while earlier batches run are packed into the next free slot, so
// their work overlaps on the device; a batch only occupies the SMs its size
// needs.  Completion is detected by polling events from the host; nothing on
// the device waits for anything.  The worker scatters each batch's counts to
// its requests' result buffers and stamps their completion time.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "qfm_common.cuh"
#include "quadfm.h"

namespace qr {
int count_kernel_params(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                        unsigned long long* queue, void* args, size_t args_bytes, cudaKernelNodeParams* p,
                        void** param_slot);
}
using qr::cuda_fail;
using qr::fail;
using qr::set_error;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    const uint8_t* pat = nullptr;     // host, offsets[0] .. offsets[m]
    const uint64_t* off = nullptr;    // host, m + 1 (any base)
    uint64_t m = 0;
    uint64_t bytes = 0;
    uint64_t* out = nullptr;          // host, m
    Clock::time_point t_submit, t_done;
    int status = 0;
    bool pinned = false;              // pat, off and out are page-locked host memory
};

struct Slot {
    uint8_t* d_pat = nullptr;
    uint64_t* d_off = nullptr;
    uint64_t* d_out = nullptr;
    unsigned long long* d_queue = nullptr;
    uint8_t* h_pat = nullptr;
    uint64_t* h_off = nullptr;
    uint64_t* h_out = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Request*> reqs;
    bool busy = false;
    bool direct = false;  // the batch was copied straight from / to the requests' buffers
    // the batch as one CUDA graph: copy in patterns, copy in offsets, reset
    // the queue, count, copy out; each batch updates the node parameters
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_pat = nullptr, n_off = nullptr, n_set = nullptr, n_ker = nullptr, n_out = nullptr;
    alignas(16) unsigned char args[512];
    void* arg_slot = nullptr;
};

}  // namespace

struct qfm_server {
    qfm_index* idx = nullptr;
    qfm_server_opts_t opt{};
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::deque<Request*> finished;   // completed, not yet polled
    uint64_t next_id = 0, submitted = 0, completed = 0, batches = 0, batched_requests = 0, graph_batches = 0;
    uint64_t in_flight_requests = 0;
    int error = QR_OK;
    std::string error_msg;
    bool stop = false;
    std::thread worker;
    Clock::time_point t0;
};

namespace {

int alloc_slot(qfm_server* sv, Slot& s) {
    const uint64_t P = sv->opt.max_batch_patterns, Bb = sv->opt.max_batch_bytes;
    QR_CUDA_TRY(cudaMalloc((void**)&s.d_pat, Bb));
    QR_CUDA_TRY(cudaMalloc((void**)&s.d_off, (P + 1) * 8));
    QR_CUDA_TRY(cudaMalloc((void**)&s.d_out, P * 8));
    QR_CUDA_TRY(cudaMalloc((void**)&s.d_queue, 16));
    QR_CUDA_TRY(cudaMallocHost((void**)&s.h_pat, Bb));
    QR_CUDA_TRY(cudaMallocHost((void**)&s.h_off, (P + 1) * 8));
    QR_CUDA_TRY(cudaMallocHost((void**)&s.h_out, P * 8));
    QR_CUDA_TRY(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    QR_CUDA_TRY(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    if (sv->opt.use_graph) {
        // nodes sized for a full slot; every batch overwrites their parameters
        QR_CUDA_TRY(cudaGraphCreate(&s.graph, 0));
        QR_CUDA_TRY(cudaGraphAddMemcpyNode1D(&s.n_pat, s.graph, nullptr, 0, s.d_pat, s.h_pat, Bb,
                                             cudaMemcpyHostToDevice));
        QR_CUDA_TRY(cudaGraphAddMemcpyNode1D(&s.n_off, s.graph, &s.n_pat, 1, s.d_off, s.h_off, (P + 1) * 8,
                                             cudaMemcpyHostToDevice));
        cudaMemsetParams ms{};
        ms.dst = s.d_queue;
        ms.elementSize = 4;
        ms.width = 4;
        ms.height = 1;
        ms.value = 0;
        QR_CUDA_TRY(cudaGraphAddMemsetNode(&s.n_set, s.graph, &s.n_off, 1, &ms));
        cudaKernelNodeParams kp{};
        int rc = qr::count_kernel_params(sv->idx, s.d_pat, s.d_off, P, s.d_out, s.d_queue, s.args, sizeof(s.args),
                                         &kp, &s.arg_slot);
        if (rc) return rc;
        QR_CUDA_TRY(cudaGraphAddKernelNode(&s.n_ker, s.graph, &s.n_set, 1, &kp));
        QR_CUDA_TRY(cudaGraphAddMemcpyNode1D(&s.n_out, s.graph, &s.n_ker, 1, s.h_out, s.d_out, P * 8,
                                             cudaMemcpyDeviceToHost));
        QR_CUDA_TRY(cudaGraphInstantiate(&s.exec, s.graph, 0));
    }
    return QR_OK;
}

// Point the slot's graph at this batch and launch it; false if the driver
// refused an update (the caller then launches the batch on the stream).
bool launch_graph(qfm_server* sv, Slot& s, const void* src_pat, uint64_t nb, const uint64_t* src_off, uint64_t np,
                  const uint8_t* d_pat, uint64_t* dst_out) {
    if (!s.exec) return false;
    cudaKernelNodeParams kp{};
    if (qr::count_kernel_params(sv->idx, d_pat, s.d_off, np, s.d_out, s.d_queue, s.args, sizeof(s.args), &kp,
                                &s.arg_slot) != QR_OK)
        return false;
    bool ok = cudaGraphExecMemcpyNodeSetParams1D(s.exec, s.n_pat, s.d_pat, src_pat, nb ? nb : 1,
                                                 cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaGraphExecMemcpyNodeSetParams1D(s.exec, s.n_off, s.d_off, src_off, (np + 1) * 8,
                                                 cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaGraphExecKernelNodeSetParams(s.exec, s.n_ker, &kp) == cudaSuccess &&
              cudaGraphExecMemcpyNodeSetParams1D(s.exec, s.n_out, dst_out, s.d_out, np * 8,
                                                 cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    return cudaGraphLaunch(s.exec, s.stream) == cudaSuccess;
}

void free_slot(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    cudaFree(s.d_pat);
    cudaFree(s.d_off);
    cudaFree(s.d_out);
    cudaFree(s.d_queue);
    cudaFreeHost(s.h_pat);
    cudaFreeHost(s.h_off);
    cudaFreeHost(s.h_out);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
}

bool is_pinned(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// r follows prev back to back in the same buffers (patterns, offsets, out).
bool adjacent(const Request* prev, const Request* r) {
    return r->pinned && r->pat == prev->pat && r->off == prev->off + prev->m && r->out == prev->out + prev->m;
}

// Pack pending requests into slot s and launch; called with sv->mu held.
int launch_batch(qfm_server* sv, Slot& s) {
    uint64_t np = 0, nb = 0;
    s.reqs.clear();
    while (!sv->pending.empty() && (int)s.reqs.size() < sv->opt.max_requests_per_batch) {
        Request* r = sv->pending.front();
        if (np + r->m > sv->opt.max_batch_patterns || nb + r->bytes > sv->opt.max_batch_bytes) break;
        sv->pending.pop_front();
        np += r->m;
        nb += r->bytes;
        s.reqs.push_back(r);
    }
    if (s.reqs.empty()) return QR_OK;
    bool direct = s.reqs[0]->pinned;
    for (size_t k = 1; k < s.reqs.size() && direct; k++) direct = adjacent(s.reqs[k - 1], s.reqs[k]);
    s.direct = direct;
    sv->in_flight_requests += s.reqs.size();
    sv->batches++;
    sv->batched_requests += s.reqs.size();
    if (sv->opt.fail_after_batches > 0 && sv->batches > (uint64_t)sv->opt.fail_after_batches)
        return fail(QR_ECUDA, "qfm_server: injected launch failure (test hook)");
    const Request* r0 = s.reqs[0];
    const uint8_t* d_pat = s.d_pat;
    if (!direct) {
        uint64_t p = 0, b = 0;
        for (Request* r : s.reqs) {
            const uint64_t base = r->off[0];
            std::memcpy(s.h_pat + b, r->pat + base, r->bytes);
            for (uint64_t k = 0; k < r->m; k++) s.h_off[p + k] = b + (r->off[k] - base);
            p += r->m;
            b += r->bytes;
        }
        s.h_off[np] = nb;
    }
    if (sv->opt.use_graph) {
        const uint64_t base = direct ? r0->off[0] : 0;
        if (launch_graph(sv, s, direct ? (const void*)(r0->pat + base) : (const void*)s.h_pat, nb,
                         direct ? r0->off : s.h_off, np, s.d_pat - base, direct ? r0->out : s.h_out)) {
            QR_CUDA_TRY(cudaEventRecord(s.done, s.stream));
            s.busy = true;
            sv->graph_batches++;
            return QR_OK;
        }
    }
    if (direct) {
        // one copy of the pattern bytes and one of the offsets, straight from
        // the requests' pinned buffers; the kernel sees the offsets as they
        // are, through a pattern pointer shifted back by offsets[0]
        const uint64_t base = r0->off[0];
        QR_CUDA_TRY(cudaMemcpyAsync(s.d_pat, r0->pat + base, nb ? nb : 1, cudaMemcpyHostToDevice, s.stream));
        QR_CUDA_TRY(cudaMemcpyAsync(s.d_off, r0->off, (np + 1) * 8, cudaMemcpyHostToDevice, s.stream));
        d_pat = s.d_pat - base;
    } else {
        QR_CUDA_TRY(cudaMemcpyAsync(s.d_pat, s.h_pat, nb ? nb : 1, cudaMemcpyHostToDevice, s.stream));
        QR_CUDA_TRY(cudaMemcpyAsync(s.d_off, s.h_off, (np + 1) * 8, cudaMemcpyHostToDevice, s.stream));
    }
    QR_CUDA_TRY(cudaMemsetAsync(s.d_queue, 0, 16, s.stream));
    int rc = qr::launch_count(sv->idx, d_pat, s.d_off, np, s.d_out, s.d_queue, s.stream, 1);
    if (rc) return rc;
    QR_CUDA_TRY(cudaMemcpyAsync(direct ? r0->out : s.h_out, s.d_out, np * 8, cudaMemcpyDeviceToHost, s.stream));
    QR_CUDA_TRY(cudaEventRecord(s.done, s.stream));
    s.busy = true;
    return QR_OK;
}

void finish_batch(qfm_server* sv, Slot& s, int status) {
    const auto now = Clock::now();
    uint64_t np = 0;
    for (Request* r : s.reqs) {
        if (status == QR_OK && !s.direct) std::memcpy(r->out, s.h_out + np, r->m * 8);
        np += r->m;
        r->status = status;
        r->t_done = now;
        sv->finished.push_back(r);
        sv->completed++;
    }
    sv->in_flight_requests -= s.reqs.size();
    s.reqs.clear();
    s.busy = false;
}

void fail_all(qfm_server* sv, int rc) {
    // called with mu held: every request not yet finished completes with rc
    if (sv->error == QR_OK) {
        sv->error = rc;
        sv->error_msg = qr_last_error();
    }
    for (Slot& s : sv->slots)
        if (!s.reqs.empty()) {
            if (s.busy) cudaStreamSynchronize(s.stream);
            finish_batch(sv, s, rc);
        }
    while (!sv->pending.empty()) {
        Request* r = sv->pending.front();
        sv->pending.pop_front();
        r->status = rc;
        r->t_done = Clock::now();
        sv->finished.push_back(r);
        sv->completed++;
    }
}

void worker_loop(qfm_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        bool progressed = false;
        // completions
        for (Slot& s : sv->slots) {
            if (!s.busy) continue;
            cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) {
                finish_batch(sv, s, QR_OK);
                progressed = true;
            } else if (e != cudaErrorNotReady) {
                qr::cuda_fail(e, "qfm_server: batch");
                fail_all(sv, QR_ECUDA);
                progressed = true;
            }
        }
        if (progressed) sv->cv_done.notify_all();
        // launches into free slots
        if (sv->error == QR_OK) {
            for (Slot& s : sv->slots) {
                if (s.busy || sv->pending.empty()) continue;
                int rc = launch_batch(sv, s);
                if (rc != QR_OK) {
                    fail_all(sv, rc);
                    sv->cv_done.notify_all();
                    break;
                }
                progressed = true;
            }
        } else if (!sv->pending.empty()) {
            fail_all(sv, sv->error);
            sv->cv_done.notify_all();
        }
        bool any_busy = false;
        for (Slot& s : sv->slots) any_busy |= s.busy;
        if (sv->stop && !any_busy && sv->pending.empty()) break;
        if (!progressed) {
            if (any_busy) {
                // batches in flight: poll again shortly
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(sv->opt.poll_us));
                lk.lock();
            } else {
                sv->cv_work.wait(lk, [&] { return sv->stop || !sv->pending.empty(); });
            }
        }
    }
}

}  // namespace

extern "C" {

int qfm_server_default_opts(qfm_server_opts_t* o) {
    if (!o) return fail(QR_EINVAL, "qfm_server_default_opts: NULL");
    o->budget_bytes = 1ull << 30;
    o->slots = 4;
    o->max_requests_per_batch = 1 << 20;
    o->max_batch_patterns = 1 << 20;
    o->max_batch_bytes = 64ull << 20;
    o->poll_us = 20;
    o->fail_after_batches = 0;
    o->use_graph = 1;
    return QR_OK;
}

int qfm_server_create(qfm_index* idx, const qfm_server_opts_t* opts, qfm_server** out) {
    if (!idx || !opts || !out) return fail(QR_EINVAL, "qfm_server_create: NULL argument");
    *out = nullptr;
    const qfm_server_opts_t& o = *opts;
    if (o.slots < 1 || o.slots > 64 || o.max_batch_patterns == 0 || o.max_batch_bytes == 0 ||
        o.max_requests_per_batch < 1 || o.poll_us < 0)
        return fail(QR_EINVAL, "qfm_server_create: invalid options");
    const uint64_t per_slot = o.max_batch_bytes + (2 * o.max_batch_patterns + 1) * 8 + 16;
    if (per_slot * (uint64_t)o.slots > o.budget_bytes)
        return fail(QR_EINVAL, "qfm_server_create: slots x batch capacity exceed the device-memory budget");
    qfm_server* sv = new qfm_server();
    sv->idx = idx;
    sv->opt = o;
    cudaGetDevice(&sv->device);
    sv->slots.resize(o.slots);
    for (Slot& s : sv->slots) {
        int rc = alloc_slot(sv, s);
        if (rc != QR_OK) {
            for (Slot& t : sv->slots) free_slot(t);
            delete sv;
            return rc;
        }
    }
    sv->t0 = Clock::now();
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return QR_OK;
}

int qfm_server_submit(qfm_server* sv, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* out,
                      uint64_t* request_id) {
    if (!sv || !offsets || (m > 0 && (!patterns || !out))) return fail(QR_EINVAL, "qfm_server_submit: NULL argument");
    if (m == 0) return fail(QR_EINVAL, "qfm_server_submit: empty request");
    if (offsets[m] < offsets[0]) return fail(QR_EINVAL, "qfm_server_submit: offsets[m] < offsets[0]");
    const uint64_t bytes = offsets[m] - offsets[0];
    if (m > sv->opt.max_batch_patterns || bytes > sv->opt.max_batch_bytes)
        return fail(QR_EINVAL, "qfm_server_submit: request larger than a batch slot");
    Request* r = new Request();
    r->pat = patterns;
    r->off = offsets;
    r->m = m;
    r->bytes = bytes;
    r->out = out;
    r->pinned = is_pinned(patterns) && is_pinned(offsets) && is_pinned(out);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            return fail(QR_EINVAL, "qfm_server_submit: server is stopping");
        }
        r->id = sv->next_id++;
        sv->submitted++;
        sv->pending.push_back(r);
    }
    sv->cv_work.notify_one();
    if (request_id) *request_id = r->id;
    return QR_OK;
}

int qfm_server_poll(qfm_server* sv, uint64_t* ids, double* latency_us, int* status, uint64_t cap, uint64_t* n_done) {
    if (!sv || !n_done || (cap > 0 && !ids)) return fail(QR_EINVAL, "qfm_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    uint64_t k = 0;
    while (k < cap && !sv->finished.empty()) {
        Request* r = sv->finished.front();
        sv->finished.pop_front();
        ids[k] = r->id;
        if (latency_us) latency_us[k] = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
        if (status) status[k] = r->status;
        delete r;
        k++;
    }
    *n_done = k;
    return QR_OK;
}

int qfm_server_drain(qfm_server* sv, double timeout_s) {
    if (!sv) return fail(QR_EINVAL, "qfm_server_drain: NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (sv->completed < sv->submitted) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && sv->completed < sv->submitted)
            return fail(QR_ETIMEOUT, "qfm_server_drain: requests still in flight at the deadline");
    }
    if (sv->error != QR_OK) {
        set_error(sv->error_msg);
        return sv->error;
    }
    return QR_OK;
}

int qfm_server_stats(qfm_server* sv, qfm_server_stats_t* st) {
    if (!sv || !st) return fail(QR_EINVAL, "qfm_server_stats: NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->pending = sv->pending.size();
    st->in_flight = sv->in_flight_requests;
    st->batches = sv->batches;
    st->mean_requests_per_batch = sv->batches ? (double)sv->batched_requests / sv->batches : 0.0;
    st->graph_batches = sv->graph_batches;
    st->error = sv->error;
    return QR_OK;
}

int qfm_server_destroy(qfm_server* sv) {
    if (!sv) return QR_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Request* r : sv->finished) delete r;
    for (Request* r : sv->pending) delete r;
    for (Slot& s : sv->slots) free_slot(s);
    delete sv;
    return QR_OK;
}

int qfm_server_replay(qfm_server* sv, const uint8_t* patterns, const uint64_t* offsets, const uint64_t* req_first,
                      uint64_t nreq, const double* arrival_s, uint64_t* out, double* latency_us, double* makespan_s) {
    if (!sv || !offsets || !req_first || !arrival_s || !out || !latency_us)
        return fail(QR_EINVAL, "qfm_server_replay: NULL argument");
    std::vector<uint64_t> ids(nreq);
    const auto start = Clock::now();
    for (uint64_t r = 0; r < nreq; r++) {
        const auto when = start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[r]));
        while (Clock::now() < when) {
            const auto left = when - Clock::now();
            if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
        }
        const uint64_t a = req_first[r], b = req_first[r + 1];
        int rc = qfm_server_submit(sv, patterns, offsets + a, b - a, out + a, &ids[r]);
        if (rc != QR_OK) return rc;
    }
    int rc = qfm_server_drain(sv, 600.0);
    const auto end = Clock::now();
    if (makespan_s) *makespan_s = std::chrono::duration<double>(end - start).count();
    // collect latencies by request id
    std::vector<uint64_t> got(4096);
    std::vector<double> lat(4096);
    std::vector<int> sts(4096);
    const uint64_t first_id = nreq ? ids[0] : 0;
    uint64_t seen = 0;
    while (seen < nreq) {
        uint64_t k = 0;
        qfm_server_poll(sv, got.data(), lat.data(), sts.data(), got.size(), &k);
        if (k == 0) break;
        for (uint64_t i = 0; i < k; i++) {
            const uint64_t r = got[i] - first_id;
            if (r < nreq) latency_us[r] = lat[i];
            if (sts[i] != QR_OK && rc == QR_OK) rc = sts[i];
        }
        seen += k;
    }
    return rc;
}

}  // extern "C"
