// Batched rank kernels over BiRank16 / QuadRank16 lines.
//
// One thread answers K independent queries: it first loads K query positions
// (coalesced, streaming), then issues the line loads of all K queries (16-byte
// vector loads, read-only path, no L1 allocation) and the superblock offsets,
// and only then does the popcounts.  The K loads in flight per thread are the
// GPU form of the paper's prefetch(q) (Sec. 3 "Prefetching"): the paper
// prefetches the line of query i + 32 while answering query i; here every
// resident thread keeps K lines in flight and the SM hides the latency across
// its warps.  Load mode 1 fetches only the 32-byte sector(s) the query needs:
// the half of the line holding its bits, plus the first 16 bytes for the
// deltas.
#include <cuda_runtime.h>

#include "qr_common.cuh"
#include "qr_rank.cuh"

namespace qr {
namespace {

template <int K, int LOAD, int KIND>
__global__ void __launch_bounds__(512) rank_kernel(RankArgs a) {
    if (a.gate && *a.gate > a.gate_limit) return;
    constexpr bool kQuad = KIND >= kQuadScalar;
    const uint64_t tile = (uint64_t)blockDim.x * K;
    uint32_t bad_flags = 0;
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < a.m; t0 += (uint64_t)gridDim.x * tile) {
        uint64_t qv[K];
        int cv[K];
        bool live[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            live[k] = i < a.m;
            qv[k] = live[k] ? ld_stream_u64(a.q + i) : 0;
            if (KIND == kBiVec || KIND == kQuadVec) cv[k] = live[k] ? (int)ld_stream_u8(a.cvec + i) : 0;
            else cv[k] = a.c;
        }
        // issue every load of the K queries before any arithmetic on them
        uint4 v0[K], va[K], vb[K];
        u64x4 r1[K], r2[K];  // load mode 4: this lane's sector of its pair's two lines
        uint32_t s1[K];
        uint4 s4[K];
        uint32_t pos[K];  // p = q - jB (sigma 2) or slot = q - jB4 + 32 (sigma 4)
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t qq = qv[k] <= a.n ? qv[k] : 0;  // out-of-range queries read line 0
            uint64_t j;
            bool upper;
            if (!kQuad) {
                j = div496(qq);
                pos[k] = (uint32_t)(qq - j * kB2);
                upper = pos[k] >= kMid2;
                s1[k] = __ldg((const uint32_t*)a.supers + (j >> 7));
            } else {
                j = div224(qq);
                pos[k] = (uint32_t)(qq - j * kB4) + 32;
                upper = pos[k] >= 128;
                if (all4<KIND>()) s4[k] = __ldg((const uint4*)a.supers + (j >> 8));
                else s1[k] = __ldg((const uint32_t*)a.supers + 4 * (j >> 8) + (cv[k] & 3));
            }
            const uint4* L = a.lines + 4 * j;
            if (LOAD == 0) {
                // whole line: four 16-byte loads (both 32-byte sectors)
                v0[k] = ld_line16(L);
                const uint4 u1 = ld_line16(L + 1), u2 = ld_line16(L + 2), u3 = ld_line16(L + 3);
                va[k] = upper ? u2 : u1;
                vb[k] = upper ? u3 : u2;
            } else if (LOAD == 1) {
                // needed sectors, 16-byte loads: lower half = quarters 0, 1 (one
                // sector); upper half = quarter 0 (deltas) + quarters 2, 3
                v0[k] = ld_line16(L);
                va[k] = ld_line16(L + (upper ? 2 : 1));
                vb[k] = upper ? ld_line16(L + 3) : make_uint4(0, 0, 0, 0);
            } else if (LOAD == 2) {
                // whole line: two 32-byte loads
                const u64x4 s0 = ld_line32(L), s1 = ld_line32(L + 2);
                v0[k] = make_uint4((uint32_t)s0.a, (uint32_t)(s0.a >> 32), (uint32_t)s0.b, (uint32_t)(s0.b >> 32));
                const uint64_t e0 = upper ? s1.a : s0.c, e1 = upper ? s1.b : s0.d;
                va[k] = make_uint4((uint32_t)e0, (uint32_t)(e0 >> 32), (uint32_t)e1, (uint32_t)(e1 >> 32));
                vb[k] = make_uint4((uint32_t)s1.c, (uint32_t)(s1.c >> 32), (uint32_t)s1.d, (uint32_t)(s1.d >> 32));
            } else if (LOAD == 4) {
                // pair-cooperative whole line: lanes 2i and 2i+1 load sector 0
                // and sector 1 of the even lane's line in one instruction (one
                // coalesced request for the 64-byte line), then the same for the
                // odd lane's line; the halves are swapped after the loads land
                const bool odd = threadIdx.x & 1;
                const uint4* P = (const uint4*)__shfl_xor_sync(0xffffffffu, (unsigned long long)L, 1);
                r1[k] = ld_line32((odd ? P : L) + 2 * odd);
                r2[k] = ld_line32((odd ? L : P) + 2 * odd);
            } else {
                // needed sectors, 32-byte loads: lower half = sector 0; upper half
                // = sector 1 + the first 16 bytes (deltas)
                if (upper) {
                    v0[k] = ld_line16(L);
                    const u64x4 s1 = ld_line32(L + 2);
                    va[k] = make_uint4((uint32_t)s1.a, (uint32_t)(s1.a >> 32), (uint32_t)s1.b, (uint32_t)(s1.b >> 32));
                    vb[k] = make_uint4((uint32_t)s1.c, (uint32_t)(s1.c >> 32), (uint32_t)s1.d, (uint32_t)(s1.d >> 32));
                } else {
                    const u64x4 s0 = ld_line32(L);
                    v0[k] = make_uint4((uint32_t)s0.a, (uint32_t)(s0.a >> 32), (uint32_t)s0.b, (uint32_t)(s0.b >> 32));
                    va[k] = make_uint4((uint32_t)s0.c, (uint32_t)(s0.c >> 32), (uint32_t)s0.d, (uint32_t)(s0.d >> 32));
                    vb[k] = make_uint4(0, 0, 0, 0);
                }
            }
        }
        if (LOAD == 4) {
            const bool odd = threadIdx.x & 1;
#pragma unroll
            for (int k = 0; k < K; k++) {
                // even lane: sector 0 = r1, sector 1 = partner's r1; odd lane:
                // sector 0 = partner's r2, sector 1 = r2
                u64x4 send = odd ? r1[k] : r2[k], recv;
                recv.a = __shfl_xor_sync(0xffffffffu, send.a, 1);
                recv.b = __shfl_xor_sync(0xffffffffu, send.b, 1);
                recv.c = __shfl_xor_sync(0xffffffffu, send.c, 1);
                recv.d = __shfl_xor_sync(0xffffffffu, send.d, 1);
                const u64x4 S0 = odd ? recv : r1[k], S1 = odd ? r2[k] : recv;
                const bool upper = kQuad ? pos[k] >= 128 : pos[k] >= kMid2;
                v0[k] = make_uint4((uint32_t)S0.a, (uint32_t)(S0.a >> 32), (uint32_t)S0.b, (uint32_t)(S0.b >> 32));
                const uint64_t e0 = upper ? S1.a : S0.c, e1 = upper ? S1.b : S0.d;
                va[k] = make_uint4((uint32_t)e0, (uint32_t)(e0 >> 32), (uint32_t)e1, (uint32_t)(e1 >> 32));
                vb[k] = make_uint4((uint32_t)S1.c, (uint32_t)(S1.c >> 32), (uint32_t)S1.d, (uint32_t)(S1.d >> 32));
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            const bool range_bad = qv[k] > a.n;
            const uint64_t w0 = lo64(v0[k]), w1 = hi64(v0[k]);
            if (!kQuad) {
                const bool upper = pos[k] >= kMid2;
                uint64_t x[4];
                if (upper) { x[0] = lo64(va[k]); x[1] = hi64(va[k]); x[2] = lo64(vb[k]); x[3] = hi64(vb[k]); }
                else { x[0] = w0; x[1] = w1; x[2] = lo64(va[k]); x[3] = hi64(va[k]); }
                const uint64_t r1 = birank_finish(s1[k], w0, x, pos[k]);
                const int c = cv[k];
                const bool sym_bad = (unsigned)c > 1u;
                uint64_t r = c == 1 ? r1 : qv[k] - r1;
                if (range_bad || sym_bad) r = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, r);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            } else {
                const bool upper = pos[k] >= 128;
                uint64_t x[4];
                if (upper) { x[0] = lo64(va[k]); x[1] = hi64(va[k]); x[2] = lo64(vb[k]); x[3] = hi64(vb[k]); }
                else { x[0] = w0; x[1] = w1; x[2] = lo64(va[k]); x[3] = hi64(va[k]); }
                if (KIND == kQuadPrefix) {
                    uint32_t s[4] = {s4[k].x, s4[k].y, s4[k].z, s4[k].w};
                    uint64_t r[4];
                    quad_finish4(s, w0, w1, x, pos[k], r);
                    uint64_t sum = 0;
#pragma unroll
                    for (int c = 0; c < 4; c++) sum += c <= a.c ? r[c] : 0;
                    if (range_bad) sum = ~0ull;
                    if (live[k]) {
                        st_stream_u64(a.out + i, sum);
                        bad_flags |= range_bad ? kStatusRange : 0u;
                    }
                } else if (KIND == kQuad4) {
                    uint32_t s[4] = {s4[k].x, s4[k].y, s4[k].z, s4[k].w};
                    uint64_t r[4];
                    quad_finish4(s, w0, w1, x, pos[k], r);
                    if (range_bad) r[0] = r[1] = r[2] = r[3] = ~0ull;
                    if (live[k]) {
                        uint64_t* o = a.out + 4 * i;
                        asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(o), "l"(r[0]), "l"(r[1]) : "memory");
                        asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(o + 2), "l"(r[2]), "l"(r[3])
                                     : "memory");
                        bad_flags |= range_bad ? kStatusRange : 0u;
                    }
                } else {
                    const int c = cv[k];
                    const bool sym_bad = (unsigned)c > 3u;
                    uint64_t r = quad_finish1(s1[k], quad_delta(w0, w1, c & 3), x, pos[k], c & 3);
                    if (range_bad || sym_bad) r = ~0ull;
                    if (live[k]) {
                        st_stream_u64(a.out + i, r);
                        bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                    }
                }
            }
        }
    }
    if (bad_flags) atomicOr(a.status, bad_flags);
}

// Sector layout (QR_LAYOUT_SECTOR): one 32-byte load per query -- the half of
// the line that holds both the query's bits and the delta to their middle.
template <int K, int KIND>
__global__ void __launch_bounds__(512) rank_sector_kernel(RankArgs a) {
    if (a.gate && *a.gate > a.gate_limit) return;
    constexpr bool kQuad = KIND >= kQuadScalar;
    const uint64_t tile = (uint64_t)blockDim.x * K;
    uint32_t bad_flags = 0;
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < a.m; t0 += (uint64_t)gridDim.x * tile) {
        uint64_t qv[K];
        int cv[K];
        bool live[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            live[k] = i < a.m;
            qv[k] = live[k] ? ld_stream_u64(a.q + i) : 0;
            if (KIND == kBiVec || KIND == kQuadVec) cv[k] = live[k] ? (int)ld_stream_u8(a.cvec + i) : 0;
            else cv[k] = a.c;
        }
        u64x4 W[K];
        uint32_t s1[K];
        uint4 s4[K];
        uint32_t r[K];  // offset inside the half: data bit (sigma 2) or char (sigma 4)
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t qq = qv[k] <= a.n ? qv[k] : 0;
            uint64_t j;
            uint32_t h;
            if (!kQuad) {
                j = div480(qq);
                const uint32_t p = (uint32_t)(qq - j * kB2s);
                h = p >= kHalf2s;
                r[k] = p - h * (uint32_t)kHalf2s;
                s1[k] = __ldg((const uint32_t*)a.supers + (j >> 7));
            } else {
                j = div192(qq);
                const uint32_t d = (uint32_t)(qq - j * kB4s);
                h = d >= kHalf4s;
                r[k] = d - h * (uint32_t)kHalf4s;
                if (all4<KIND>()) s4[k] = __ldg((const uint4*)a.supers + (j >> 8));
                else s1[k] = __ldg((const uint32_t*)a.supers + 4 * (j >> 8) + (cv[k] & 3));
            }
            W[k] = ld_line32(a.lines + 4 * j + 2 * h);
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            const bool range_bad = qv[k] > a.n;
            if (!kQuad) {
                const uint64_t r1 = birank_sector_finish(s1[k], W[k], r[k]);
                const int c = cv[k];
                const bool sym_bad = (unsigned)c > 1u;
                uint64_t res = c == 1 ? r1 : qv[k] - r1;
                if (range_bad || sym_bad) res = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, res);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            } else if (KIND == kQuadPrefix) {
                const uint32_t s[4] = {s4[k].x, s4[k].y, s4[k].z, s4[k].w};
                uint64_t res[4];
                quad_sector_finish4(s, W[k], r[k], res);
                uint64_t sum = 0;
#pragma unroll
                for (int c = 0; c < 4; c++) sum += c <= a.c ? res[c] : 0;
                if (range_bad) sum = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, sum);
                    bad_flags |= range_bad ? kStatusRange : 0u;
                }
            } else if (KIND == kQuad4) {
                const uint32_t s[4] = {s4[k].x, s4[k].y, s4[k].z, s4[k].w};
                uint64_t res[4];
                quad_sector_finish4(s, W[k], r[k], res);
                if (range_bad) res[0] = res[1] = res[2] = res[3] = ~0ull;
                if (live[k]) {
                    uint64_t* o = a.out + 4 * i;
                    asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(o), "l"(res[0]), "l"(res[1]) : "memory");
                    asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(o + 2), "l"(res[2]), "l"(res[3])
                                 : "memory");
                    bad_flags |= range_bad ? kStatusRange : 0u;
                }
            } else {
                const int c = cv[k];
                const bool sym_bad = (unsigned)c > 3u;
                uint64_t res = quad_sector_finish1(s1[k], W[k], r[k], c & 3);
                if (range_bad || sym_bad) res = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, res);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            }
        }
    }
    if (bad_flags) atomicOr(a.status, bad_flags);
}

// Dependent queries (latency mode): every thread follows one chain, each
// query position derived from the previous answer, so only one line per chain
// is ever in flight.  Whole warps run the chains of 32 consecutive starts, so
// that on the paper layout the two lanes of a pair can load the two sectors
// of both their lines in two instructions: one request (one line fill) per
// query, as in load mode 4.  The sector layout needs one sector per query.
template <bool QUAD, bool SECTOR>
__device__ __forceinline__ uint64_t rank_one(const RankArgs& a, uint64_t q, int c) {
    if (SECTOR) {
        if (!QUAD) {
            const uint64_t j = div480(q);
            const uint32_t p = (uint32_t)(q - j * kB2s), h = p >= kHalf2s;
            const uint32_t s = __ldg((const uint32_t*)a.supers + (j >> 7));
            const u64x4 W = ld_line32(a.lines + 4 * j + 2 * h);
            const uint64_t r1 = birank_sector_finish(s, W, p - h * (uint32_t)kHalf2s);
            return c == 1 ? r1 : q - r1;
        }
        const uint64_t j = div192(q);
        const uint32_t d = (uint32_t)(q - j * kB4s), h = d >= kHalf4s;
        const uint32_t s = __ldg((const uint32_t*)a.supers + 4 * (j >> 8) + c);
        const u64x4 W = ld_line32(a.lines + 4 * j + 2 * h);
        return quad_sector_finish1(s, W, d - h * (uint32_t)kHalf4s, c);
    }
    constexpr uint32_t kAll = 0xffffffffu;
    const uint64_t j = QUAD ? div224(q) : div496(q);
    const uint32_t pos = QUAD ? (uint32_t)(q - j * kB4) + 32 : (uint32_t)(q - j * kB2);
    const bool upper = QUAD ? pos >= 128 : pos >= kMid2;
    const uint32_t s = QUAD ? __ldg((const uint32_t*)a.supers + 4 * (j >> 8) + c)
                            : __ldg((const uint32_t*)a.supers + (j >> 7));
    const uint4* L = a.lines + 4 * j;
    const bool odd = threadIdx.x & 1;
    const uint4* P = (const uint4*)__shfl_xor_sync(kAll, (unsigned long long)L, 1);
    const u64x4 r1 = ld_line32((odd ? P : L) + 2 * odd);  // even: own sector 0; odd: partner's sector 1
    const u64x4 r2 = ld_line32((odd ? L : P) + 2 * odd);  // even: partner's sector 0; odd: own sector 1
    const u64x4 send = odd ? r1 : r2;
    u64x4 recv;
    recv.a = __shfl_xor_sync(kAll, send.a, 1);
    recv.b = __shfl_xor_sync(kAll, send.b, 1);
    recv.c = __shfl_xor_sync(kAll, send.c, 1);
    recv.d = __shfl_xor_sync(kAll, send.d, 1);
    const u64x4 S0 = odd ? recv : r1, S1 = odd ? r2 : recv;
    const u64x4 H = upper ? S1 : S0;
    const uint64_t x[4] = {H.a, H.b, H.c, H.d};
    if (!QUAD) {
        const uint64_t r = birank_finish(s, S0.a, x, pos);
        return c == 1 ? r : q - r;
    }
    return quad_finish1(s, quad_delta(S0.a, S0.b, c), x, pos, c);
}

// a.q = chain starts (a.m chains), a.out[2k] = final position, a.out[2k+1] =
// last rank; a.c = symbol; steps per chain in `steps`.  A start > n runs a
// chain from 0 (its lanes still take part in the pair loads) and reports
// UINT64_MAX.
template <bool QUAD, bool SECTOR>
__global__ void __launch_bounds__(256) rank_chain_kernel(RankArgs a, uint64_t steps) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); base < a.m; base += stride) {
        const uint64_t k = base + lane;
        const bool live = k < a.m;
        uint64_t q = live ? a.q[k] : 0, r = 0;
        const bool bad = q > a.n;
        if (bad) q = 0;
        for (uint64_t t = 0; t < steps; t++) {
            r = rank_one<QUAD, SECTOR>(a, q, a.c);
            if (t + 1 < steps) q = chain_next(q, r, a.n);
        }
        if (live) {
            a.out[2 * k] = bad ? ~0ull : q;
            a.out[2 * k + 1] = bad ? ~0ull : r;
            if (bad) atomicOr(a.status, kStatusRange);
        }
    }
}

// ---------------------------------------------------------------- launch table
template <int K, int KIND>
KernelFn pick_load(int load) {
    switch (load) {
        case 0: return rank_kernel<K, 0, KIND>;
        case 1: return rank_kernel<K, 1, KIND>;
        case 2: return rank_kernel<K, 2, KIND>;
        case 3: return rank_kernel<K, 3, KIND>;
        case 4: return rank_kernel<K, 4, KIND>;
        default: return nullptr;
    }
}

template <int KIND>
KernelFn pick(int k, int load) {
    switch (k) {
        case 1: return pick_load<1, KIND>(load);
        case 2: return pick_load<2, KIND>(load);
        case 4: return pick_load<4, KIND>(load);
        case 8: return pick_load<8, KIND>(load);
        default: return nullptr;
    }
}

template <int KIND>
KernelFn pick_sector(int k) {
    switch (k) {
        case 1: return rank_sector_kernel<1, KIND>;
        case 2: return rank_sector_kernel<2, KIND>;
        case 4: return rank_sector_kernel<4, KIND>;
        case 8: return rank_sector_kernel<8, KIND>;
        default: return nullptr;
    }
}

KernelFn pick_kind(int kind, int k, int load, int layout) {
    if (layout == QR_LAYOUT_LINE128) return pick_line_kind(kind, k);
    if (inline_layout(layout)) return pick_in32_kind(kind, k, layout);
    const bool sector = layout == QR_LAYOUT_SECTOR;
    if (sector) {
        switch (kind) {
            case kBiScalar: return pick_sector<kBiScalar>(k);
            case kBiVec: return pick_sector<kBiVec>(k);
            case kQuadScalar: return pick_sector<kQuadScalar>(k);
            case kQuadVec: return pick_sector<kQuadVec>(k);
            case kQuad4: return pick_sector<kQuad4>(k);
            case kQuadPrefix: return pick_sector<kQuadPrefix>(k);
            default: return nullptr;
        }
    }
    switch (kind) {
        case kBiScalar: return pick<kBiScalar>(k, load);
        case kBiVec: return pick<kBiVec>(k, load);
        case kQuadScalar: return pick<kQuadScalar>(k, load);
        case kQuadVec: return pick<kQuadVec>(k, load);
        case kQuad4: return pick<kQuad4>(k, load);
        case kQuadPrefix: return pick<kQuadPrefix>(k, load);
        default: return nullptr;
    }
}

unsigned resident_grid(KernelFn fn, int threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (unsigned)(per_sm * device_props().sms);
}

// ---------------------------------------------------------------- gather probe
__device__ __forceinline__ uint64_t probe_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// V = 16-byte quarters per record, W = bytes per load: 16 or 32 (each lane
// reads its own record), 128 (128-byte records read quad-cooperatively as the
// 128-byte line rank kernels do: lane s of a quad loads sector s of the four
// records of the quad in four instructions, then an XOR reduce-scatter gives
// every lane the digest of its own record).
template <int K, int V, int W>
__global__ void __launch_bounds__(1024) probe_kernel(const uint4* __restrict__ buf, uint64_t nrec, uint64_t m,
                                                     uint64_t seed, uint64_t* __restrict__ out) {
    constexpr uint32_t kAll = 0xffffffffu;
    const uint64_t tile = (uint64_t)blockDim.x * K;
    constexpr int kLoads = W == 128 ? 4 : W == 32 && V >= 2 ? V / 2 : V;
    const int sub = threadIdx.x & 3;
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < m; t0 += (uint64_t)gridDim.x * tile) {
        uint64_t v[K][kLoads];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            const uint64_t r = mulhi64(probe_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ull), nrec);
#pragma unroll
            for (int u = 0; u < kLoads; u++) {
                if (W == 128) {
                    const uint64_t ru = __shfl_sync(kAll, (unsigned long long)r, u, 4);
                    const u64x4 x = ld_line32(buf + ru * 8 + 2 * sub);
                    v[k][u] = x.a ^ x.b ^ x.c ^ x.d;
                } else if (W == 32 && V >= 2) {
                    const u64x4 x = ld_line32(buf + r * V + 2 * u);
                    v[k][u] = x.a ^ x.b ^ x.c ^ x.d;
                } else {
                    const uint4 x = ld_line16(buf + r * V + u);
                    v[k][u] = lo64(x) ^ hi64(x);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            uint64_t d = 0;
            if (W == 128) {
                const bool hi2 = sub & 2, hi1 = sub & 1;
                const uint64_t a0 = (hi2 ? v[k][2] : v[k][0]) ^
                                    __shfl_xor_sync(kAll, (unsigned long long)(hi2 ? v[k][0] : v[k][2]), 2, 4);
                const uint64_t a1 = (hi2 ? v[k][3] : v[k][1]) ^
                                    __shfl_xor_sync(kAll, (unsigned long long)(hi2 ? v[k][1] : v[k][3]), 2, 4);
                d = (hi1 ? a1 : a0) ^ __shfl_xor_sync(kAll, (unsigned long long)(hi1 ? a0 : a1), 1, 4);
            } else {
#pragma unroll
                for (int u = 0; u < kLoads; u++) d ^= v[k][u];
            }
            if (i < m) st_stream_u64(out + i, d);
        }
    }
}

// L2 probe: random 64-byte records (two 32-byte loads each) of a buffer small
// enough to stay in L2.  MODE 0: every thread issues four independent
// records per round, their data folded into one digest (the random-request
// throughput of L2).  MODE 1: every thread runs one chain; a round reads two
// records whose indices come from the chain state, and the next state mixes
// both records' data, as the two interval ends of an LF step depend on the
// step before (the latency-bound rate of such chains at this occupancy).
template <int MODE>
__global__ void __launch_bounds__(256) probe_l2_kernel(const uint4* __restrict__ buf, uint64_t nrec, uint32_t rounds,
                                                       uint64_t seed, uint64_t nthreads, uint64_t* __restrict__ out) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    uint64_t st = probe_mix(seed + (t + 1) * 0x9E3779B97F4A7C15ull);
    uint64_t d = 0;
    for (uint32_t r = 0; r < rounds; r++) {
        if (MODE == 0) {
            u64x4 x[4][2];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint64_t rec = mulhi64(probe_mix(st + (uint64_t)k * 0xD1B54A32D192ED03ull), nrec);
                x[k][0] = ld_line32(buf + 4 * rec);
                x[k][1] = ld_line32(buf + 4 * rec + 2);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) d ^= x[k][0].a ^ x[k][0].d ^ x[k][1].b ^ x[k][1].c;
            st = probe_mix(st + 1);
        } else {
            const uint64_t ra = mulhi64(st, nrec), rb = mulhi64(probe_mix(st ^ 0xD1B54A32D192ED03ull), nrec);
            const u64x4 a0 = ld_line32(buf + 4 * ra), a1 = ld_line32(buf + 4 * ra + 2);
            const u64x4 b0 = ld_line32(buf + 4 * rb), b1 = ld_line32(buf + 4 * rb + 2);
            const uint64_t v = a0.a ^ a0.d ^ a1.b ^ a1.c ^ b0.b ^ b0.c ^ b1.a ^ b1.d;
            d ^= v;
            st = probe_mix(st + v + 1);
        }
    }
    st_stream_u64(out + t, d);
}

}  // namespace

int launch_rank(const qr_index* idx, const uint64_t* q, const uint8_t* cvec, int c, uint64_t m, uint64_t* out,
                int rank4, cudaStream_t s) {
    if (m == 0) return QR_OK;
    if (region_supported(idx, rank4) && idx->batch_mode != QR_BATCH_DIRECT &&
        (idx->batch_mode == QR_BATCH_REGIONS ? m < (1ull << 32) : region_auto(idx, m))) {
        // the automatic rule adds a device-side probe: a clustered (e.g.
        // sorted) batch is answered by the direct kernels after all
        const DirectLaunch direct = [&](const unsigned long long* count, unsigned long long limit) {
            return launch_direct(idx, q, cvec, c, m, out, rank4, s, count, limit);
        };
        cudaEvent_t* marks = idx->region_timing ? (cudaEvent_t*)idx->region_ev : nullptr;
        const int rc = launch_rank_regions(idx, q, cvec, c, m, out, rank4, s, marks,
                                           idx->batch_mode == QR_BATCH_AUTO ? &direct : nullptr);
        if (rc != QR_ENOMEM) return rc;  // without scratch memory the direct kernels answer the batch
    }
    return launch_direct(idx, q, cvec, c, m, out, rank4, s, nullptr, 0);
}

int launch_direct(const qr_index* idx, const uint64_t* q, const uint8_t* cvec, int c, uint64_t m, uint64_t* out,
                  int rank4, cudaStream_t s, const unsigned long long* gate, unsigned long long gate_limit) {
    int kind;
    if (idx->sigma == 2) kind = cvec ? kBiVec : kBiScalar;
    else kind = rank4 == 2 ? kQuadPrefix : rank4 ? kQuad4 : (cvec ? kQuadVec : kQuadScalar);
    qr_tuning_t t = idx->tune;
    // under the gate the batch is clustered (e.g. sorted): neighbouring
    // threads then share lines, and two queries in flight per thread beat
    // more (measured on sorted 2^28-query batches: K = 2 191 Gq/s, K = 4 156,
    // K = 8 83), so the tuning found on the uniform batch is not reused
    if (gate && t.queries_per_thread > 2) t.queries_per_thread = 2;
    KernelFn fn = pick_kind(kind, t.queries_per_thread, t.load_mode, idx->layout);
    if (!fn) return fail(QR_EINVAL, "no rank kernel for this tuning");
    RankArgs a{idx->lines, idx->supers, idx->n, q, cvec, c, m, out, idx->status, gate, gate_limit};
    const uint64_t tiles = (m + (uint64_t)t.block_threads * t.queries_per_thread - 1) /
                           ((uint64_t)t.block_threads * t.queries_per_thread);
    uint64_t grid = t.grid_blocks > 0 ? (uint64_t)t.grid_blocks : resident_grid(fn, t.block_threads);
    if (grid > tiles) grid = tiles;
    fn<<<(unsigned)grid, t.block_threads, 0, s>>>(a);
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

int launch_chain(const qr_index* idx, const uint64_t* q0, uint64_t nchains, uint64_t steps, int c, uint64_t* out,
                 cudaStream_t s) {
    if (nchains == 0) return QR_OK;
    RankArgs a{idx->lines, idx->supers, idx->n, q0, nullptr, c, nchains, out, idx->status, nullptr, 0};
    const bool quad = idx->sigma == 4, sector = idx->layout == QR_LAYOUT_SECTOR;
    ChainFn fn = idx->layout == QR_LAYOUT_LINE128 ? pick_chain_line(quad)
                 : inline_layout(idx->layout)
                     ? pick_chain_in32(quad, idx->layout)
                     : quad ? (sector ? rank_chain_kernel<true, true> : rank_chain_kernel<true, false>)
                            : (sector ? rank_chain_kernel<false, true> : rank_chain_kernel<false, false>);
    uint64_t grid = (nchains + 255) / 256;
    const uint64_t cap = (uint64_t)device_props().sms * 8;
    if (grid > cap) grid = cap;
    fn<<<(unsigned)grid, 256, 0, s>>>(a, steps);
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

int launch_probe(const void* buf, uint64_t nrec, int bytes, int load_bytes, uint64_t m, uint64_t seed, uint64_t* out,
                 int k, int threads, cudaStream_t s) {
    if (m == 0) return QR_OK;
    void (*fn)(const uint4*, uint64_t, uint64_t, uint64_t, uint64_t*) = nullptr;
#define QR_PROBE_CASE(KK, VV)                                                            \
    if (k == KK && bytes == 16 * VV && load_bytes == 16) fn = probe_kernel<KK, VV, 16>; \
    if (k == KK && bytes == 16 * VV && load_bytes == 32 && VV >= 2) fn = probe_kernel<KK, VV, 32>; \
    if (k == KK && bytes == 128 && VV == 8 && load_bytes == 128) fn = probe_kernel<KK, 8, 128>;
    QR_PROBE_CASE(1, 1) QR_PROBE_CASE(1, 2) QR_PROBE_CASE(1, 4) QR_PROBE_CASE(1, 8)
    QR_PROBE_CASE(2, 1) QR_PROBE_CASE(2, 2) QR_PROBE_CASE(2, 4) QR_PROBE_CASE(2, 8)
    QR_PROBE_CASE(4, 1) QR_PROBE_CASE(4, 2) QR_PROBE_CASE(4, 4) QR_PROBE_CASE(4, 8)
    QR_PROBE_CASE(8, 1) QR_PROBE_CASE(8, 2) QR_PROBE_CASE(8, 4)
#undef QR_PROBE_CASE
    if (!fn) return fail(QR_EINVAL, "qr_probe_gather: unsupported (bytes, queries_per_thread)");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint64_t tiles = (m + (uint64_t)threads * k - 1) / ((uint64_t)threads * k);
    uint64_t grid = (uint64_t)per_sm * device_props().sms;
    if (grid > tiles) grid = tiles;
    fn<<<(unsigned)grid, threads, 0, s>>>((const uint4*)buf, nrec, m, seed, out);
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

int launch_probe_l2(const void* buf, uint64_t nrec, int mode, uint64_t nthreads, uint32_t rounds, uint64_t seed,
                    uint64_t* out, int threads, cudaStream_t s) {
    if (nthreads == 0) return QR_OK;
    const uint64_t grid = (nthreads + threads - 1) / threads;
    if (grid > 0x7fffffffull) return fail(QR_EINVAL, "qr_probe_l2: too many threads");
    auto fn = mode == 0 ? probe_l2_kernel<0> : probe_l2_kernel<1>;
    fn<<<(unsigned)grid, threads, 0, s>>>((const uint4*)buf, nrec, rounds, seed, nthreads, out);
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

}  // namespace qr
