// Batched rank over the inline layouts (paper Sec. 3.1 BiRank32 and
// BiRank32x2, Sec. 4.1 QuadRank32 and QuadRank24_8): the value inlined in the
// line (or half-line) plus the line's L0 entry gives the rank at the middle
// (QuadRank24_8: at char 64, or at char 192 with its 8-bit step), and the
// bits or characters between the query and that point are counted as in the
// 16-bit layouts (Sec. 3 Eq. 1, Sec. 4 rank1 and rank_4).
//
// BiRank32x2 keeps each 32-byte half self-contained: one sector per query.
// BiRank32 and the two sigma-4 layouts need the whole 64-byte line (the value
// sits in the first sector, most data in the second): the two lanes of a pair
// load the
// two sectors of both their lines in two instructions, so each line is one
// request and one DRAM fill, as in load mode 4 of the paper layout.
//
// Variants (template V): kV32 = BiRank32 / QuadRank32, kVX2 = BiRank32x2,
// kV24 = QuadRank24_8 (sigma 4 only).
#include <cuda_runtime.h>

#include "qr_common.cuh"
#include "qr_rank.cuh"

namespace qr {
namespace {

constexpr uint32_t kAll = 0xffffffffu;
constexpr int kV32 = 0, kVX2 = 1, kV24 = 2;

// The two sectors of this lane's line, loaded with its pair partner: lane 2i
// and lane 2i + 1 load sector 0 and sector 1 of lane 2i's line in one
// instruction, then those of lane 2i + 1's line, and exchange halves.  Every
// lane of the warp must call it.
__device__ __forceinline__ void pair_line(const uint4* L, u64x4& S0, u64x4& S1) {
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
    S0 = odd ? recv : r1;
    S1 = odd ? r2 : recv;
}

// One query (chains): the rank of symbol c at q.  QUAD: sigma 4.  Every lane
// of the warp must call it.
template <bool QUAD, int V>
__device__ __forceinline__ uint64_t rank_one_in32(const RankArgs& a, uint64_t q, int c) {
    const uint64_t* l0 = (const uint64_t*)a.supers;
    if (!QUAD && V == kVX2) {
        const uint64_t j = div448(q);
        const uint32_t p = (uint32_t)(q - j * kB2x), h = p >= kHalf2x;
        const u64x4 W = ld_line32(a.lines + 4 * j + 2 * h);
        const uint64_t r1 = in32x2_finish(__ldg(l0 + (j >> kL0Shift)), W, p - h * (uint32_t)kHalf2x);
        return c == 1 ? r1 : q - r1;
    }
    const uint64_t j = QUAD ? div192(q) : div480(q);
    const uint32_t d = (uint32_t)(q - j * (QUAD ? kB4w : kB2w));
    u64x4 S0, S1;
    pair_line(a.lines + 4 * j, S0, S1);
    if (QUAD && V == kV24) return quad24_finish1(__ldg(l0 + 4 * (j >> kL0Shift24) + c), S0, S1, d, c);
    if (QUAD) return quad32_finish1(__ldg(l0 + 4 * (j >> kL0Shift) + c), S0, S1, d, c);
    const uint64_t r1 = in32_bi_finish(__ldg(l0 + (j >> kL0Shift)), S0, S1, d);
    return c == 1 ? r1 : q - r1;
}

template <int K, int KIND, int V>
__global__ void __launch_bounds__(512) rank_in32_kernel(RankArgs a) {
    if (a.gate && *a.gate > a.gate_limit) return;
    constexpr bool kQuad = KIND >= kQuadScalar;
    constexpr bool X2 = V == kVX2;
    constexpr int kShift = V == kV24 ? kL0Shift24 : kL0Shift;
    const uint64_t* l0 = (const uint64_t*)a.supers;
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
        // every load of the K queries before any arithmetic on them
        u64x4 S0[K], S1[K];
        uint64_t base[K];   // L0 entry (of the query's symbol)
        uint4 b4lo[K], b4hi[K];  // rank_4 / prefix_rank: the four L0 entries
        uint32_t pos[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t qq = qv[k] <= a.n ? qv[k] : 0;  // out-of-range queries read line 0
            if (!kQuad && X2) {
                const uint64_t j = div448(qq);
                const uint32_t p = (uint32_t)(qq - j * kB2x), h = p >= kHalf2x;
                pos[k] = p - h * (uint32_t)kHalf2x;
                base[k] = __ldg(l0 + (j >> kL0Shift));
                S0[k] = ld_line32(a.lines + 4 * j + 2 * h);
            } else {
                const uint64_t j = kQuad ? div192(qq) : div480(qq);
                pos[k] = (uint32_t)(qq - j * (kQuad ? kB4w : kB2w));
                if (!kQuad) base[k] = __ldg(l0 + (j >> kL0Shift));
                else if (all4<KIND>()) {
                    const uint4* e = (const uint4*)(l0 + 4 * (j >> kShift));
                    b4lo[k] = __ldg(e);
                    b4hi[k] = __ldg(e + 1);
                } else {
                    base[k] = __ldg(l0 + 4 * (j >> kShift) + (cv[k] & 3));
                }
                pair_line(a.lines + 4 * j, S0[k], S1[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            const bool range_bad = qv[k] > a.n;
            if (!kQuad) {
                const uint64_t r1 = X2 ? in32x2_finish(base[k], S0[k], pos[k])
                                       : in32_bi_finish(base[k], S0[k], S1[k], pos[k]);
                const int c = cv[k];
                const bool sym_bad = (unsigned)c > 1u;
                uint64_t r = c == 1 ? r1 : qv[k] - r1;
                if (range_bad || sym_bad) r = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, r);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            } else if (all4<KIND>()) {
                const uint64_t b[4] = {lo64(b4lo[k]), hi64(b4lo[k]), lo64(b4hi[k]), hi64(b4hi[k])};
                uint64_t r[4];
                if (V == kV24) quad24_finish4(b, S0[k], S1[k], pos[k], r);
                else quad32_finish4(b, S0[k], S1[k], pos[k], r);
                if (KIND == kQuadPrefix) {
                    uint64_t sum = 0;
#pragma unroll
                    for (int c = 0; c < 4; c++) sum += c <= a.c ? r[c] : 0;
                    if (range_bad) sum = ~0ull;
                    if (live[k]) {
                        st_stream_u64(a.out + i, sum);
                        bad_flags |= range_bad ? kStatusRange : 0u;
                    }
                } else {
                    if (range_bad) r[0] = r[1] = r[2] = r[3] = ~0ull;
                    if (live[k]) {
                        uint64_t* o = a.out + 4 * i;
                        st_stream_v2u64(o, r[0], r[1]);
                        st_stream_v2u64(o + 2, r[2], r[3]);
                        bad_flags |= range_bad ? kStatusRange : 0u;
                    }
                }
            } else {
                const int c = cv[k];
                const bool sym_bad = (unsigned)c > 3u;
                uint64_t r = V == kV24 ? quad24_finish1(base[k], S0[k], S1[k], pos[k], c & 3)
                                       : quad32_finish1(base[k], S0[k], S1[k], pos[k], c & 3);
                if (range_bad || sym_bad) r = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, r);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            }
        }
    }
    if (bad_flags) atomicOr(a.status, bad_flags);
}

// Dependent queries (latency mode) over the inline layouts; whole warps run
// the chains of 32 consecutive starts (the pair loads need both lanes).  A
// start > n runs a chain from 0 and reports UINT64_MAX.
template <bool QUAD, int V>
__global__ void __launch_bounds__(256) rank_chain_in32_kernel(RankArgs a, uint64_t steps) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); b < a.m; b += stride) {
        const uint64_t k = b + lane;
        const bool live = k < a.m;
        uint64_t q = live ? a.q[k] : 0, r = 0;
        const bool bad = q > a.n;
        if (bad) q = 0;
        for (uint64_t t = 0; t < steps; t++) {
            r = rank_one_in32<QUAD, V>(a, q, a.c);
            if (t + 1 < steps) q = chain_next(q, r, a.n);
        }
        if (live) {
            a.out[2 * k] = bad ? ~0ull : q;
            a.out[2 * k + 1] = bad ? ~0ull : r;
            if (bad) atomicOr(a.status, kStatusRange);
        }
    }
}

template <int KIND, int V>
KernelFn pick_k(int k) {
    switch (k) {
        case 1: return rank_in32_kernel<1, KIND, V>;
        case 2: return rank_in32_kernel<2, KIND, V>;
        case 4: return rank_in32_kernel<4, KIND, V>;
        case 8: return rank_in32_kernel<8, KIND, V>;
        default: return nullptr;
    }
}

template <int V>
KernelFn pick_quad(int kind, int k) {
    switch (kind) {
        case kQuadScalar: return pick_k<kQuadScalar, V>(k);
        case kQuadVec: return pick_k<kQuadVec, V>(k);
        case kQuad4: return pick_k<kQuad4, V>(k);
        case kQuadPrefix: return pick_k<kQuadPrefix, V>(k);
        default: return nullptr;
    }
}

}  // namespace

KernelFn pick_in32_kind(int kind, int k, int layout) {
    if (layout == QR_LAYOUT_INLINE32X2) {
        switch (kind) {
            case kBiScalar: return pick_k<kBiScalar, kVX2>(k);
            case kBiVec: return pick_k<kBiVec, kVX2>(k);
            default: return nullptr;  // BiRank32x2 is sigma 2 only
        }
    }
    if (layout == QR_LAYOUT_INLINE24_8) return pick_quad<kV24>(kind, k);  // sigma 4 only
    switch (kind) {
        case kBiScalar: return pick_k<kBiScalar, kV32>(k);
        case kBiVec: return pick_k<kBiVec, kV32>(k);
        default: return pick_quad<kV32>(kind, k);
    }
}

ChainFn pick_chain_in32(bool quad, int layout) {
    if (layout == QR_LAYOUT_INLINE24_8) return quad ? rank_chain_in32_kernel<true, kV24> : nullptr;
    if (quad) return rank_chain_in32_kernel<true, kV32>;
    return layout == QR_LAYOUT_INLINE32X2 ? rank_chain_in32_kernel<false, kVX2>
                                          : rank_chain_in32_kernel<false, kV32>;
}

}  // namespace qr
