// Approximate counting over the QuadFm index: occurrences of a pattern with
// at most k substituted characters, by backtracking backward search.  This
// is the use of rank_4 the paper names (Sec. 1: returning all four ranks at
// once serves approximate pattern matching in an FM-index): at every node of
// the search the interval [lo, hi) is extended by all four characters at
// once, from rank_4(lo) and rank_4(hi) (Sec. 4), and the children other than
// the pattern's own character are explored while mismatches remain.
//
// Every string P' within Hamming distance k of P is reached exactly once, so
// the sum of their interval sizes is the number of text positions where P
// matches with at most k substitutions.  The search order is depth-first
// with one frame per mismatch level (at most k + 1 frames per lane): a frame
// walks the pattern right to left by exact steps and, before each step,
// opens a child frame for every substituted character whose interval is not
// empty.  Lanes take patterns from a device work queue as in qfm_count.
#include "qfm_common.cuh"
#include "quadfm.h"

namespace qr {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxK = 3;  // at most 3 substitutions: the frames stay in a few hundred bytes

// rank(q, c) for all four c from the half-line holding q (stored BWT: the $
// row counts as code 0).
__device__ __forceinline__ void fm_rank4_line(const FmLine& f, const uint4 s4, uint32_t slot, uint32_t r[4]) {
    const QuadHalf32 h = quad_half32(f.x, slot);
    uint32_t nl = 0, nh = 0, n3 = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t L = ~h.nl[i] & h.m[i], H = ~h.nh[i] & h.m[i];
        nl += __popc(L);
        nh += __popc(H);
        n3 += __popc(L & H);
    }
    const bool upper = slot >= 128;
    const uint32_t nm = upper ? slot - 128 : 128 - slot;
    const uint32_t n[4] = {nm - nl - nh + n3, nl - n3, nh - n3, n3};
    const uint32_t d0 = lo32(f.d0), d1 = lo32(f.d1);
    const uint32_t dl[4] = {d0 & 0xFFFFu, d0 >> 16, d1 & 0xFFFFu, d1 >> 16};
    const uint32_t sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint32_t mid = (sv[c] << kShift4) + dl[c];
        r[c] = upper ? mid + n[c] : mid - n[c];
    }
}

// The four children of [lo, hi): [C[c] + rank(lo, c), C[c] + rank(hi, c)),
// less the $ row for c = 0.  lo and hi share the fetch when they fall in one
// half-line.
__device__ __forceinline__ void fm_children(const FmView& v, uint32_t lo, uint32_t hi, uint32_t clo[4],
                                            uint32_t chi[4]) {
    const uint32_t jl = div224_32(lo), jh = div224_32(hi);
    const uint32_t sl = lo - jl * (uint32_t)kB4 + 32, sh = hi - jh * (uint32_t)kB4 + 32;
    const bool ul = sl >= 128, uh = sh >= 128;
    const uint4 s4l = __ldg(v.supers + (jl >> 8));
    const uint4 s4h = jl >> 8 == jh >> 8 ? s4l : __ldg(v.supers + (jh >> 8));
    const FmLine fl = fm_fetch<false>(v.lines + 4 * (uint64_t)jl, ul, 0);
    const FmLine fh = (jl == jh && ul == uh) ? fl : fm_fetch<false>(v.lines + 4 * (uint64_t)jh, uh, 0);
    uint32_t rl[4], rh[4];
    fm_rank4_line(fl, s4l, sl, rl);
    fm_rank4_line(fh, s4h, sh, rh);
    const uint32_t d = (uint32_t)v.dollar;
    rl[0] -= lo > d ? 1u : 0u;
    rh[0] -= hi > d ? 1u : 0u;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint32_t Cc = (uint32_t)v.C[c];
        clo[c] = Cc + rl[c];
        chi[c] = Cc + rh[c];
    }
}

// One mismatch level of the depth-first search.
struct Frame {
    int32_t pos;       // next pattern index to consume (right to left); -1: done
    uint32_t lo, hi;   // interval of the suffix matched so far
    uint32_t clo[4], chi[4];
    int32_t cnext;     // next substituted character to try at pos (children known)
    bool expanded;     // children of [lo, hi) computed for pos
};

struct ApproxArgs {
    FmView v;
    const uint8_t* __restrict__ pat;
    const uint64_t* __restrict__ off;
    uint64_t m;
    uint64_t* __restrict__ out;
    unsigned long long* queue;
    uint32_t* status;
    uint32_t k;
    uint32_t chunk;
};

__global__ void __launch_bounds__(kThreads) count_approx_kernel(ApproxArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t total = a.m ? a.off[a.m] : 0;
    uint64_t pool_next = 0, pool_end = 0;
    bool drained = false, active = false;
    uint64_t id = 0, start = 0, count = 0;
    int d = 0;  // current frame
    Frame F[kMaxK + 1];
    uint32_t bad = 0;
    while (true) {
        // ---- refill idle lanes from the work queue
        const unsigned need = __ballot_sync(0xffffffffu, !active);
        if (need && !drained) {
            const uint32_t cnt = __popc(need), r = __popc(need & lt_mask);
            const uint64_t avail = pool_end - pool_next;
            uint64_t base = 0;
            if (avail < cnt) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(a.queue, (unsigned long long)a.chunk);
                base = __shfl_sync(0xffffffffu, (unsigned long long)b, 0);
            }
            if (!active) {
                id = r < avail ? pool_next + r : base + (r - avail);
                if (id < a.m) {
                    start = a.off[id];
                    const uint64_t end = a.off[id + 1];
                    bool ok = end >= start && end <= total;
                    for (uint64_t i = start; ok && i < end; i++) ok = a.pat[i] <= 3;
                    if (!ok) {
                        a.out[id] = 0;  // malformed: offsets out of order or a byte > 3
                        bad |= kStatusBadSym;
                    } else {
                        d = 0;
                        F[0].pos = (int32_t)(end - start) - 1;
                        F[0].lo = 0;
                        F[0].hi = (uint32_t)a.v.nrows;
                        F[0].expanded = false;
                        count = 0;
                        active = true;
                    }
                }
            }
            if (avail < cnt) {
                pool_next = base + (cnt - avail);
                pool_end = base + a.chunk;
                if (base >= a.m) drained = true;
            } else {
                pool_next += cnt;
            }
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (drained || pool_next >= a.m) break;
            continue;
        }
        // ---- advance the search until the next expansion (or its end)
        bool expand = false;
        while (active) {
            Frame& f = F[d];
            if (!f.expanded) {
                if (f.lo >= f.hi || f.pos < 0) {
                    if (f.lo < f.hi) count += f.hi - f.lo;  // a full string P' matched
                    if (--d < 0) {
                        st_stream_u64(a.out + id, count);
                        active = false;
                    }
                    continue;
                }
                expand = true;
                break;
            }
            const int pc = a.pat[start + f.pos];
            if (d < (int)a.k) {
                while (f.cnext < 4 && (f.cnext == pc || f.clo[f.cnext] >= f.chi[f.cnext])) ++f.cnext;
                if (f.cnext < 4) {
                    const int c = f.cnext++;
                    Frame& g = F[d + 1];
                    g.pos = f.pos - 1;
                    g.lo = f.clo[c];
                    g.hi = f.chi[c];
                    g.expanded = false;
                    ++d;
                    continue;
                }
            }
            // substitutions at pos done: the exact step
            f.lo = f.clo[pc];
            f.hi = f.chi[pc];
            --f.pos;
            f.expanded = false;
        }
        // ---- expansions of all lanes together
        if (expand) {
            Frame& f = F[d];
            fm_children(a.v, f.lo, f.hi, f.clo, f.chi);
            f.cnext = 0;
            f.expanded = true;
        }
    }
    if (bad) atomicOr(a.status, bad);
}

}  // namespace

int launch_count_approx(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint32_t k, uint64_t* out,
                        unsigned long long* queue, cudaStream_t s) {
    ApproxArgs a;
    fm_view(idx, &a.v);
    a.pat = pat;
    a.off = off;
    a.m = m;
    a.out = out;
    a.queue = queue;
    a.status = idx->status;
    a.k = k;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, count_approx_kernel, kThreads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    uint64_t grid = (uint64_t)per_sm * device_props().sms;
    a.chunk = m >= grid * (kThreads / 32) * 64 ? 64 : 32;
    const uint64_t blocks_needed = ((m + a.chunk - 1) / a.chunk + kThreads / 32 - 1) / (kThreads / 32);
    if (grid > blocks_needed) grid = blocks_needed;
    if (grid == 0) grid = 1;
    count_approx_kernel<<<(unsigned)grid, kThreads, 0, s>>>(a);
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

}  // namespace qr

using namespace qr;

extern "C" int qfm_count_approx(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m,
                                int max_mismatches, uint64_t* out, void* stream) {
    if (!idx) return fail(QR_EINVAL, "qfm_count_approx: index is NULL");
    if (max_mismatches < 0 || max_mismatches > kMaxK) return fail(QR_EINVAL, "qfm_count_approx: k must be 0..3");
    if (m == 0) return QR_OK;
    if (!patterns || !offsets || !out) return fail(QR_EINVAL, "qfm_count_approx: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* queue = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&queue, 16, s));
    cudaError_t e = cudaMemsetAsync(queue, 0, 16, s);
    int rc = QR_OK;
    // no substitution allowed: the exact count (prefix table, one rank per end)
    if (e == cudaSuccess)
        rc = max_mismatches == 0
                 ? launch_count(idx, patterns, offsets, m, out, queue, s, 1)
                 : launch_count_approx(idx, patterns, offsets, m, (uint32_t)max_mismatches, out, queue, s);
    cudaFreeAsync(queue, s);
    if (e != cudaSuccess) return cuda_fail(e, "qfm_count_approx: queue reset");
    return rc;
}
