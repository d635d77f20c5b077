// Count-only backward search over the QuadFm index (paper App. D).
//
// qfm_count: one persistent launch.  Every warp takes pattern ids from a
// device work queue (an atomic counter) in chunks of 64 (32 for small
// batches), keeps one search per lane, and refills its idle lanes in groups
// of at least 8, so the lanes of a warp stay busy despite uneven pattern
// lengths and early mismatches.  This is
// the GPU form of the paper's query_batch: a batch of active searches where
// finished ones are swapped out and the rest take one rank + LF step per pass.
//
// qfm_count_stepwise: the plain form, one launch per search step over every
// pattern (a table-lookup launch, then max-steps launches).
#include <mutex>

#include "qfm_common.cuh"
#include "quadfm.h"

namespace qr {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kChunkMax = 64;  // pattern ids taken from the queue at once per warp
// A warp refills its lanes once at least this many are idle (or all are): the
// refill path costs the whole warp the same instructions for 1 lane as for 8,
// and a lane finishes a search about every 26 steps, so refilling per finished
// lane would run it on almost every step.  Measured on the 10^7-pattern
// workload: 1 -> 2.70, 4 -> 3.13, 8 -> 3.27, 16 -> 2.96 G patterns/s.
constexpr uint32_t kRefillMin = 8;

struct CountArgs {
    FmView v;
    const uint8_t* __restrict__ pat;
    const uint64_t* __restrict__ off;
    uint64_t m;
    uint64_t* __restrict__ out;
    unsigned long long* queue;
    uint32_t* status;
    uint32_t chunk;  // ids per queue grab: 64, or 32 when the batch is too small to fill the grid
    uint32_t strands;  // 1: patterns as given; 2: also their reverse complements (ids m..2m-1)
    uint64_t* lohi;    // optional: the final interval [lo, hi) of search id at lohi[2 id], lohi[2 id + 1]
};

// Start a search: the interval of the last 8 chars from the table (or the full
// interval for shorter patterns).  With rc the searched string is the reverse
// complement of p (char k = 3 - p[len-1-k]), so its last 8 chars are the
// complements of p[7], p[6], ..., p[0].  Returns false for a malformed pattern.
__device__ __forceinline__ bool fm_start(const FmView& v, const uint8_t* __restrict__ p, uint64_t len, bool rc,
                                         uint64_t& lo, uint64_t& hi, int64_t& i) {
    if (len >= (uint64_t)kQfmK) {
        uint32_t w = 0, badc = 0;
#pragma unroll
        for (int d = 0; d < kQfmK; d++) {
            const uint32_t raw = rc ? p[kQfmK - 1 - d] : p[len - kQfmK + d];
            badc |= raw;
            w = (w << 2) | ((rc ? 3 - raw : raw) & 3);
        }
        if (badc > 3) return false;
        lo = __ldg(v.table + 2 * w);
        hi = __ldg(v.table + 2 * w + 1);
        i = (int64_t)len - kQfmK - 1;
    } else {
        lo = 0;
        hi = v.nrows;
        i = (int64_t)len - 1;
    }
    return true;
}

// A lane reads its pattern through a 16-byte register window: one aligned
// vector load per 16 characters instead of one byte load per step.  `cur` is
// the byte offset (from pat) of the next char, moving by `dir` per step (-1
// for a pattern, +1 for its reverse complement); `k` is cur's index in the
// window, kNoWindow when cur is outside it.  The window is only loaded when
// the whole aligned chunk lies inside the pattern buffer [pat, pat + total);
// otherwise the byte is loaded alone.
constexpr int32_t kNoWindow = 1 << 20;  // stays outside [0, 16) under +-1 steps

struct PatWindow {
    uint4 w;
    uint64_t lo = 0;      // byte offset (from pat) of the window start
    bool valid = false;
    int32_t k = kNoWindow;
};

// Index of byte offset p in the current window (at the start of a search).
__device__ __forceinline__ int32_t window_index(const PatWindow& win, uint64_t p) {
    return win.valid && p >= win.lo && p - win.lo < 16 ? (int32_t)(p - win.lo) : kNoWindow;
}

template <bool STREAM>
__device__ __forceinline__ int pattern_char(const uint8_t* __restrict__ pat, uint64_t total, uint64_t p, PatWindow& win,
                                            uint64_t pol_first) {
    if ((uint32_t)win.k >= 16u) {
        const uint64_t a = p - (((uintptr_t)(pat + p)) & 15);  // aligned chunk start, as an offset
        if (a <= p && a + 16 <= total) {
            win.w = STREAM ? ld_line16_hint((const uint4*)(pat + a), pol_first) : __ldg((const uint4*)(pat + a));
            win.lo = a;
            win.valid = true;
            win.k = (int32_t)(p - a);
        } else {
            return pat[p];
        }
    }
    const uint32_t k = (uint32_t)win.k;
    const uint32_t word = k < 8 ? (k < 4 ? win.w.x : win.w.y) : (k < 12 ? win.w.z : win.w.w);
    return (int)__byte_perm(word, 0u, 0x4440u | (k & 3));
}

template <int POLICY, int STRANDS>
__global__ void __launch_bounds__(kThreads, 4) count_persistent(CountArgs a) {
    constexpr bool kKeep = POLICY == kFmPolicyKeepIndex || POLICY == kFmPolicyKeepIndexOnly;
    constexpr bool kFirst = POLICY == kFmPolicyKeepIndex;  // pattern / offset stream evict-first
    constexpr bool kBoth = STRANDS == 2;
    const uint64_t pol_last = kKeep ? l2_policy_evict_last() : 0;
    const uint64_t pol_first = kFirst ? l2_policy_evict_first() : 0;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t total = a.m ? a.off[a.m] : 0;  // bytes of the pattern buffer
    const uint64_t work = a.m * STRANDS;           // search ids: [0, m) forward, [m, 2m) reverse complement
    PatWindow win;
    // warp-local pool of pattern ids [pool_next, pool_end)
    uint64_t pool_next = 0, pool_end = 0;
    bool drained = false;  // the queue has no ids left for this warp
    bool active = false;
    uint64_t id = 0, cur = 0;  // cur: byte offset of the next char to read
    uint32_t lo = 0, hi = 0;   // BWT rows < 2^32
    int64_t i = -1;
    bool rc = false;
    int dir = -1;
    uint32_t bad = 0;
    while (true) {
        // ---- refill lanes whose search ended
        const unsigned need = __ballot_sync(0xffffffffu, !active);
        if (need && !drained && (__popc(need) >= kRefillMin || need == 0xffffffffu)) {
            const uint32_t cnt = __popc(need);
            const uint32_t r = __popc(need & lt_mask);
            const uint64_t avail = pool_end - pool_next;
            uint64_t base = 0;
            if (avail < cnt) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(a.queue, (unsigned long long)a.chunk);
                base = __shfl_sync(0xffffffffu, (unsigned long long)b, 0);
            }
            if (!active) {
                id = r < avail ? pool_next + r : base + (r - avail);
                if (id < work) {
                    rc = kBoth && id >= a.m;
                    const uint64_t pid = rc ? id - a.m : id;
                    const uint64_t start = kFirst ? ld_u64_hint(a.off + pid, pol_first) : a.off[pid];
                    const uint64_t end = kFirst ? ld_u64_hint(a.off + pid + 1, pol_first) : a.off[pid + 1];
                    const uint64_t len = end - start;
                    uint64_t lo0 = 0, hi0 = 0;
                    if (end < start || end > total || !fm_start(a.v, a.pat + start, len, rc, lo0, hi0, i)) {
                        a.out[id] = 0;  // malformed: offsets out of order or a byte > 3
                        if (a.lohi) a.lohi[2 * id] = a.lohi[2 * id + 1] = 0;
                        bad |= kStatusBadSym;
                    } else {
                        lo = (uint32_t)lo0;
                        hi = (uint32_t)hi0;
                        // char i of the searched string: p[i], or 3 - p[len-1-i] for the reverse complement
                        cur = rc ? start + (len - 1 - (uint64_t)i) : start + (uint64_t)i;
                        dir = rc ? 1 : -1;
                        win.k = window_index(win, cur);
                        active = true;
                    }
                }
            }
            if (avail < cnt) {
                pool_next = base + (cnt - avail);
                pool_end = base + a.chunk;
                if (base >= work) drained = true;
            } else {
                pool_next += cnt;
            }
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (drained || pool_next >= work) break;
            continue;
        }
        // ---- one LF step for every active lane
        if (active) {
            if (i >= 0 && lo < hi) {
                const int raw = pattern_char<kFirst>(a.pat, total, cur, win, pol_first);
                cur += dir;
                win.k += dir;
                const int c = rc && raw <= 3 ? 3 - raw : raw;
                if (c > 3) {
                    a.out[id] = 0;
                    if (a.lohi) a.lohi[2 * id] = a.lohi[2 * id + 1] = 0;
                    bad |= kStatusBadSym;
                    active = false;
                } else {
                    fm_lf_pair<kKeep>(a.v, lo, hi, c, pol_last);
                    --i;
                }
            }
            if (active && (i < 0 || lo >= hi)) {
                st_stream_u64(a.out + id, hi > lo ? (uint64_t)(hi - lo) : 0);
                if (a.lohi) {
                    a.lohi[2 * id] = lo;
                    a.lohi[2 * id + 1] = hi > lo ? hi : lo;
                }
                active = false;
            }
        }
    }
    if (bad) atomicOr(a.status, bad);
}

// ---- stepwise baseline
struct StepState {
    uint64_t lo, hi;
    int64_t i;  // next pattern index to consume; -2 = finished
};

__global__ void step_init(CountArgs a, StepState* __restrict__ st, unsigned long long* __restrict__ max_steps) {
    uint64_t local_max = 0;
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < a.m; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = a.off[k], e = a.off[k + 1];
        StepState x;
        if (e < s || e > a.off[a.m] || !fm_start(a.v, a.pat + s, e - s, false, x.lo, x.hi, x.i)) {
            a.out[k] = 0;
            atomicOr(a.status, kStatusBadSym);
            x.i = -2;
        } else {
            local_max = max(local_max, (uint64_t)(x.i + 1));
        }
        st[k] = x;
    }
    atomicMax(max_steps, (unsigned long long)local_max);
}

__global__ void step_once(CountArgs a, StepState* __restrict__ st) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < a.m; k += (uint64_t)gridDim.x * blockDim.x) {
        StepState x = st[k];
        if (x.i == -2) continue;
        if (x.i >= 0 && x.lo < x.hi) {
            const int c = a.pat[a.off[k] + x.i];
            if (c > 3) {
                a.out[k] = 0;
                atomicOr(a.status, kStatusBadSym);
                st[k].i = -2;
                continue;
            }
            x.lo = fm_lf(a.v, x.lo, c);
            x.hi = fm_lf(a.v, x.hi, c);
            --x.i;
        }
        if (x.i < 0 || x.lo >= x.hi) {
            a.out[k] = x.hi > x.lo ? x.hi - x.lo : 0;
            x.i = -2;
        }
        st[k] = x;
    }
}

using CountFn = void (*)(CountArgs);

CountFn count_fn(int policy, int strands) {
    if (policy == kFmPolicyKeepIndex) return strands == 2 ? count_persistent<1, 2> : count_persistent<1, 1>;
    if (policy == kFmPolicyKeepIndexOnly) return strands == 2 ? count_persistent<2, 2> : count_persistent<2, 1>;
    return strands == 2 ? count_persistent<0, 2> : count_persistent<0, 1>;
}

unsigned persistent_grid(int policy, int strands = 1) {
    static thread_local int per_sm[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int& k = per_sm[policy >= 0 && policy <= 2 ? policy : 1][strands == 2];
    if (k == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, count_fn(policy, strands), kThreads, 0);
        if (e != cudaSuccess || k < 1) k = 1;
    }
    return (unsigned)(k * device_props().sms);
}

}  // namespace

int launch_count(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                 unsigned long long* queue, cudaStream_t s, int strands, uint64_t* lohi) {
    CountArgs a;
    a.strands = strands == 2 ? 2 : 1;
    a.lohi = lohi;
    fm_view(idx, &a.v);
    a.pat = pat;
    a.off = off;
    a.m = m;
    a.out = out;
    a.queue = queue;
    a.status = idx->status;
    uint64_t grid = persistent_grid(idx->policy, a.strands);
    const uint64_t work = m * a.strands;
    // one queue grab per warp of 64 ids when there are enough searches to
    // keep every resident warp busy; smaller batches take 32 (one per lane)
    a.chunk = work >= (uint64_t)grid * (kThreads / 32) * kChunkMax * 2 ? kChunkMax : 32;
    uint64_t warps_needed = (work + a.chunk - 1) / a.chunk;
    const uint64_t blocks_needed = (warps_needed + kThreads / 32 - 1) / (kThreads / 32);
    if (grid > blocks_needed) grid = blocks_needed;
    if (grid == 0) grid = 1;
    count_fn(idx->policy, a.strands)<<<(unsigned)grid, kThreads, 0, s>>>(a);
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

// Kernel-node parameters of the same launch, for callers that put it in a CUDA
// graph: `args` (at least sizeof(CountArgs) bytes, 16-byte aligned) receives
// the argument block that p->kernelParams points to.
int count_kernel_params(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                        unsigned long long* queue, void* args, size_t args_bytes, cudaKernelNodeParams* p,
                        void** param_slot) {
    if (args_bytes < sizeof(CountArgs)) return fail(QR_EINVAL, "count_kernel_params: argument block too small");
    CountArgs* a = (CountArgs*)args;
    fm_view(idx, &a->v);
    a->pat = pat;
    a->off = off;
    a->m = m;
    a->out = out;
    a->queue = queue;
    a->status = idx->status;
    a->strands = 1;
    a->lohi = nullptr;
    uint64_t grid = persistent_grid(idx->policy);
    a->chunk = m >= grid * (kThreads / 32) * kChunkMax * 2 ? kChunkMax : 32;
    const uint64_t warps_needed = (m + a->chunk - 1) / a->chunk;
    const uint64_t blocks_needed = (warps_needed + kThreads / 32 - 1) / (kThreads / 32);
    if (grid > blocks_needed) grid = blocks_needed;
    if (grid == 0) grid = 1;
    *param_slot = a;
    p->func = (void*)count_fn(idx->policy, 1);
    p->gridDim = dim3((unsigned)grid);
    p->blockDim = dim3(kThreads);
    p->sharedMemBytes = 0;
    p->kernelParams = param_slot;
    p->extra = nullptr;
    return QR_OK;
}

int launch_count_stepwise(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                          cudaStream_t s) {
    CountArgs a;
    fm_view(idx, &a.v);
    a.pat = pat;
    a.off = off;
    a.m = m;
    a.out = out;
    a.queue = nullptr;
    a.status = idx->status;
    a.lohi = nullptr;
    StepState* st = nullptr;
    unsigned long long* mx = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&st, m * sizeof(StepState), s));
    cudaError_t e = cudaMallocAsync((void**)&mx, 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, 8, s);
    uint64_t blocks = (m + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)device_props().sms * 16;
    if (blocks > cap) blocks = cap;
    unsigned long long steps = 0;
    if (e == cudaSuccess) {
        step_init<<<(unsigned)blocks, kThreads, 0, s>>>(a, st, mx);
        e = cudaMemcpyAsync(&steps, mx, 8, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (unsigned long long t = 0; e == cudaSuccess && t < steps + 1; t++) {
        step_once<<<(unsigned)blocks, kThreads, 0, s>>>(a, st);
        e = cudaGetLastError();
    }
    cudaFreeAsync(st, s);
    cudaFreeAsync(mx, s);
    if (e != cudaSuccess) return cuda_fail(e, "qfm_count_stepwise");
    return QR_OK;
}

}  // namespace qr

// ---------------------------------------------------------------------------
// qfm_count_noalloc: qfm_count for callers that cannot allocate device memory.
//
// The persistent kernel's only scratch is its work-queue counter.  qfm_count
// takes it from the stream-ordered pool; this variant keeps it in the static
// device array below instead, so a call makes no cudaMalloc, cudaMallocAsync,
// cudaFree or other allocating call.  The array is part of the library image:
// every GPU that loads the library holds its 256 bytes until the process
// exits.  In host code the name g_noalloc_scratch is only a host-side stand-in
// for the device array, so its device address is looked up once per device
// with cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned long long g_noalloc_scratch[32];  // 256 bytes

namespace qr {
namespace {

constexpr size_t kNoallocScratchBytes = sizeof(g_noalloc_scratch);
constexpr size_t kNoallocQueueBytes = 16;  // one work-queue counter (+ padding)
constexpr int kNoallocMaxDevices = 64;

std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the static scratch on the current device (looked up on
// the first call per device, with that device current).
int noalloc_scratch(unsigned long long** out) {
    int dev = 0;
    QR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(QR_EINVAL, "qfm_count_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "qfm_count_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = (unsigned long long*)p;
    }
    *out = g_noalloc_ptr[dev];
    return QR_OK;
}

}  // namespace
}  // namespace qr

extern "C" int qfm_count_noalloc(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m,
                                 uint64_t* out, void* stream) {
    using namespace qr;
    if (!idx) return fail(QR_EINVAL, "qfm_count_noalloc: index is NULL");
    if (m > 0 && (!patterns || !offsets || !out)) return fail(QR_EINVAL, "qfm_count_noalloc: NULL buffer");
    if (m == 0) return QR_OK;
    // the scratch a call needs: one work-queue counter, whatever m is
    if (kNoallocQueueBytes > kNoallocScratchBytes)
        return fail(QR_EINVAL, "qfm_count_noalloc: scratch need exceeds the 256-byte static array");
    unsigned long long* queue = nullptr;
    int rc = noalloc_scratch(&queue);
    if (rc != QR_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's counter: start this call's queue at 0
    QR_CUDA_TRY(cudaMemsetAsync(queue, 0, kNoallocQueueBytes, s));
    return launch_count(idx, patterns, offsets, m, out, queue, s, 1);
}
