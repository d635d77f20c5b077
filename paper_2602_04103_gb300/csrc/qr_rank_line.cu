// Batched rank over the 128-byte line layout (QR_LAYOUT_LINE128).
//
// The four lanes of a quad answer their four queries together.  For each
// query r of the quad every lane loads its sector (32 bytes) of query r's
// line: four lanes, one instruction, one request and one 128-byte fill per
// query.  Each lane computes its signed part of the answer -- plus or minus
// the ones (or chars) of the query's range that fall in its sector, plus the
// delta on the lane holding sector 0 -- and a reduce-scatter over the quad
// (3 shuffles per value) leaves lane r with the sum for query r.
//
// Range counts without range masks: the range runs from the query position X
// to the line's middle M (where the delta is anchored), so the bits of the
// range are those under prefix(X) XOR prefix(M), both prefix masks of the
// line's bit order.  prefix(M) restricted to a lane's sector is a constant of
// the lane; prefix(X) over a 32-bit word is one funnel shift.  The sign is
// X >= M (count added) or X < M (count subtracted), as in Sec. 3 of the
// paper.
#include <cuda_runtime.h>

#include "qr_common.cuh"
#include "qr_rank.cuh"

namespace qr {
namespace {

constexpr uint32_t kAll = 0xffffffffu;

// Sum over the quad of v[r] lands in lane r (values of any integer type).
template <typename T>
__device__ __forceinline__ T quad_reduce_scatter(const T v[4], int sub) {
    const bool hi2 = sub & 2, hi1 = sub & 1;
    // lanes sub ^ 2: keep the two indices of this lane's half, pass the others
    const T s0 = hi2 ? v[0] : v[2], s1 = hi2 ? v[1] : v[3];
    const T k0 = hi2 ? v[2] : v[0], k1 = hi2 ? v[3] : v[1];
    const T a0 = k0 + (T)__shfl_xor_sync(kAll, s0, 2, 4);
    const T a1 = k1 + (T)__shfl_xor_sync(kAll, s1, 2, 4);
    // lanes sub ^ 1: keep index sub
    return (hi1 ? a1 : a0) + (T)__shfl_xor_sync(kAll, hi1 ? a0 : a1, 1, 4);
}

// sigma 2 (BiRank16 on 1008-bit lines): line bit 16 + p holds data offset p,
// the delta counts the ones before data offset 504 = line bit 520.  Lane sub
// holds line bits [256 sub, 256 sub + 256) as words w[0..7] of 32 bits.  The
// 16 delta bits lie under both prefix masks and cancel.
struct BiLane {
    uint32_t mid[8];   // prefix mask of line bit 520 over each word of the sector
    int32_t base;      // 256 sub
};
__device__ __forceinline__ BiLane bi_lane(int sub) {
    BiLane L;
    L.base = 256 * sub;
#pragma unroll
    for (int i = 0; i < 8; i++) L.mid[i] = low32(16 + (int32_t)kMid2L - L.base - 32 * i);
    return L;
}
__device__ __forceinline__ uint32_t bi_part(const BiLane& L, const u64x4& W, int32_t x) {
    const uint32_t w[8] = {lo32(W.a), hi32(W.a), lo32(W.b), hi32(W.b), lo32(W.c), hi32(W.c), lo32(W.d), hi32(W.d)};
    const int32_t xs = x - L.base;
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) cnt += __popc(w[i] & (low32(xs - 32 * i) ^ L.mid[i]));
    return cnt;
}

// sigma 4 (QuadRank16 on 480-char lines): word 0 = the four deltas, word 1 =
// chars 448..479 (~low bits | ~high bits << 32), words 2 + 2g / 3 + 2g =
// ~low / ~high bits of chars 64 g .. 64 g + 63; the deltas count chars before
// char 240.  A lane sees four half-groups of 32 chars, each a pair of 32-bit
// words (~low, ~high) and the char index of its first char:
//   sub 0:  chars 448.. (word 1), none, chars 0.., chars 32.. (words 2, 3)
//   sub k:  chars 128k - 64 .., 128k - 32 .. (words 4k, 4k+1),
//           chars 128k .., 128k + 32 .. (words 4k+2, 4k+3).
struct QuadLane {
    uint32_t mid[4];   // prefix mask of char 240 over each half-group
    int32_t base[4];   // first char of each half-group (>= 480: empty)
    bool s0;
};
__device__ __forceinline__ QuadLane quad_lane(int sub) {
    QuadLane L;
    L.s0 = sub == 0;
    const int32_t b = 128 * sub;
    L.base[0] = L.s0 ? 448 : b - 64;
    L.base[1] = L.s0 ? 480 : b - 32;
    L.base[2] = b;
    L.base[3] = b + 32;
#pragma unroll
    for (int j = 0; j < 4; j++) L.mid[j] = low32((int32_t)kMid4L - L.base[j]);
    return L;
}
// The (~low, ~high) word pairs of the four half-groups.
__device__ __forceinline__ void quad_words(const QuadLane& L, const u64x4& W, uint32_t nl[4], uint32_t nh[4]) {
    const uint64_t a = L.s0 ? (W.b & 0xFFFFFFFFull) : W.a;
    const uint64_t b = L.s0 ? (W.b >> 32) : W.b;
    nl[0] = lo32(a); nh[0] = lo32(b);
    nl[1] = hi32(a); nh[1] = hi32(b);
    nl[2] = lo32(W.c); nh[2] = lo32(W.d);
    nl[3] = hi32(W.c); nh[3] = hi32(W.d);
}
// chars equal to c in this lane's part of the range
__device__ __forceinline__ uint32_t quad_part1(const QuadLane& L, const u64x4& W, int32_t x, int c) {
    uint32_t nl[4], nh[4];
    quad_words(L, W, nl, nh);
    const uint32_t cl = 0u - (uint32_t)(c & 1), ch = 0u - (uint32_t)(c >> 1);
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t m = low32(x - L.base[j]) ^ L.mid[j];
        cnt += __popc((nl[j] ^ cl) & (nh[j] ^ ch) & m);
    }
    return cnt;
}
// |low bits|, |high bits|, |both| of the chars in this lane's part of the range
__device__ __forceinline__ void quad_part4(const QuadLane& L, const u64x4& W, int32_t x, int32_t& pl, int32_t& ph,
                                          int32_t& p3) {
    uint32_t nl[4], nh[4];
    quad_words(L, W, nl, nh);
    uint32_t a = 0, b = 0, c = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t m = low32(x - L.base[j]) ^ L.mid[j];
        const uint32_t lo = ~nl[j] & m, hi = ~nh[j] & m;
        a += __popc(lo);
        b += __popc(hi);
        c += __popc(lo & hi);
    }
    pl = (int32_t)a;
    ph = (int32_t)b;
    p3 = (int32_t)c;
}

template <int K, int KIND>
__global__ void __launch_bounds__(512) rank_line_kernel(RankArgs a) {
    constexpr bool kQuad = KIND >= kQuadScalar;
    const int sub = threadIdx.x & 3;
    const BiLane bl = bi_lane(sub);
    const QuadLane ql = quad_lane(sub);
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
        uint32_t pos[K];
        uint32_t s1[K];
        uint4 s4[K];
        u64x4 W[K][4];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t qq = qv[k] <= a.n ? qv[k] : 0;  // out-of-range queries read line 0
            uint64_t j;
            if (!kQuad) {
                j = div1008(qq);
                pos[k] = (uint32_t)(qq - j * kB2L);
                s1[k] = __ldg((const uint32_t*)a.supers + (j >> 5));
            } else {
                j = div480(qq);
                pos[k] = (uint32_t)(qq - j * kB4L);
                if (all4<KIND>()) s4[k] = __ldg((const uint4*)a.supers + (j >> 6));
                else s1[k] = __ldg((const uint32_t*)a.supers + 4 * (j >> 6) + (cv[k] & 3));
            }
            const unsigned long long L = (unsigned long long)(a.lines + 8 * j);
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const uint4* Lr = (const uint4*)__shfl_sync(kAll, L, r, 4);
                W[k][r] = ld_line32(Lr + 2 * sub);
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            uint64_t res[4] = {0, 0, 0, 0};
            if (!kQuad) {
                int32_t part[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const uint32_t pr = __shfl_sync(kAll, pos[k], r, 4);
                    const int32_t cnt = (int32_t)bi_part(bl, W[k][r], 16 + (int32_t)pr);
                    part[r] = (pr >= kMid2L ? cnt : -cnt) + (sub == 0 ? (int32_t)(W[k][r].a & 0xFFFFull) : 0);
                }
                // delta +- count of the own query: rank(q) - 2^11 s >= 0
                res[0] = ((uint64_t)s1[k] << kShift2) + (uint64_t)(int64_t)quad_reduce_scatter(part, sub);
            } else if (!all4<KIND>()) {
                int32_t part[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const uint32_t pr = __shfl_sync(kAll, pos[k], r, 4);
                    const int cr = __shfl_sync(kAll, cv[k], r, 4) & 3;
                    const int32_t cnt = (int32_t)quad_part1(ql, W[k][r], (int32_t)pr, cr);
                    part[r] = (pr >= kMid4L ? cnt : -cnt) +
                              (sub == 0 ? (int32_t)((W[k][r].a >> (16 * cr)) & 0xFFFFull) : 0);
                }
                res[0] = ((uint64_t)s1[k] << kShift4) + (uint64_t)(int64_t)quad_reduce_scatter(part, sub);
            } else {
                int32_t pl[4], ph[4], p3[4];
                unsigned long long pd[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const uint32_t pr = __shfl_sync(kAll, pos[k], r, 4);
                    quad_part4(ql, W[k][r], (int32_t)pr, pl[r], ph[r], p3[r]);
                    pd[r] = sub == 0 ? W[k][r].a : 0;  // the four deltas of line r
                }
                const uint32_t nl = (uint32_t)quad_reduce_scatter(pl, sub);
                const uint32_t nh = (uint32_t)quad_reduce_scatter(ph, sub);
                const uint32_t n3 = (uint32_t)quad_reduce_scatter(p3, sub);
                const uint64_t d0 = quad_reduce_scatter(pd, sub);
                const bool upper = pos[k] >= kMid4L;
                const uint32_t nm = upper ? pos[k] - (uint32_t)kMid4L : (uint32_t)kMid4L - pos[k];
                const uint32_t nc[4] = {nm - nl - nh + n3, nl - n3, nh - n3, n3};
                const uint32_t sv[4] = {s4[k].x, s4[k].y, s4[k].z, s4[k].w};
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const uint64_t mid = ((uint64_t)sv[c] << kShift4) + ((d0 >> (16 * c)) & 0xFFFFull);
                    res[c] = upper ? mid + nc[c] : mid - nc[c];
                }
            }
            const bool range_bad = qv[k] > a.n;
            if (!kQuad) {
                const int c = cv[k];
                const bool sym_bad = (unsigned)c > 1u;
                uint64_t out = c == 1 ? res[0] : qv[k] - res[0];
                if (range_bad || sym_bad) out = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, out);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            } else if (KIND == kQuadPrefix) {
                uint64_t sum = 0;
#pragma unroll
                for (int c = 0; c < 4; c++) sum += c <= a.c ? res[c] : 0;
                if (range_bad) sum = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, sum);
                    bad_flags |= range_bad ? kStatusRange : 0u;
                }
            } else if (KIND == kQuad4) {
                if (range_bad) res[0] = res[1] = res[2] = res[3] = ~0ull;
                if (live[k]) {
                    uint64_t* o = a.out + 4 * i;
                    asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(o), "l"(res[0]), "l"(res[1]) : "memory");
                    asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(o + 2), "l"(res[2]), "l"(res[3])
                                 : "memory");
                    bad_flags |= range_bad ? kStatusRange : 0u;
                }
            } else {
                const bool sym_bad = (unsigned)cv[k] > 3u;
                uint64_t out = res[0];
                if (range_bad || sym_bad) out = ~0ull;
                if (live[k]) {
                    st_stream_u64(a.out + i, out);
                    bad_flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                }
            }
        }
    }
    if (bad_flags) atomicOr(a.status, bad_flags);
}

// Dependent queries on 128-byte lines: the quad's four chains take their
// steps together, each step reading the four lines quad-cooperatively.
template <bool QUAD>
__device__ __forceinline__ uint64_t rank_line_one(const RankArgs& a, const BiLane& bl, const QuadLane& ql, int sub,
                                                  uint64_t q, int c) {
    uint64_t j;
    uint32_t pos, s;
    if (!QUAD) {
        j = div1008(q);
        pos = (uint32_t)(q - j * kB2L);
        s = __ldg((const uint32_t*)a.supers + (j >> 5));
    } else {
        j = div480(q);
        pos = (uint32_t)(q - j * kB4L);
        s = __ldg((const uint32_t*)a.supers + 4 * (j >> 6) + c);
    }
    const unsigned long long L = (unsigned long long)(a.lines + 8 * j);
    u64x4 W[4];
#pragma unroll
    for (int r = 0; r < 4; r++) W[r] = ld_line32((const uint4*)__shfl_sync(kAll, L, r, 4) + 2 * sub);
    int32_t part[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const uint32_t pr = __shfl_sync(kAll, pos, r, 4);
        if (!QUAD) {
            const int32_t cnt = (int32_t)bi_part(bl, W[r], 16 + (int32_t)pr);
            part[r] = (pr >= kMid2L ? cnt : -cnt) + (sub == 0 ? (int32_t)(W[r].a & 0xFFFFull) : 0);
        } else {
            const int32_t cnt = (int32_t)quad_part1(ql, W[r], (int32_t)pr, c);
            part[r] = (pr >= kMid4L ? cnt : -cnt) + (sub == 0 ? (int32_t)((W[r].a >> (16 * c)) & 0xFFFFull) : 0);
        }
    }
    const int64_t sum = quad_reduce_scatter(part, sub);
    if (!QUAD) {
        const uint64_t r1 = ((uint64_t)s << kShift2) + (uint64_t)sum;
        return c == 1 ? r1 : q - r1;
    }
    return ((uint64_t)s << kShift4) + (uint64_t)sum;
}

template <bool QUAD>
__global__ void __launch_bounds__(256) rank_chain_line_kernel(RankArgs a, uint64_t steps) {
    const int sub = threadIdx.x & 3;
    const BiLane bl = bi_lane(sub);
    const QuadLane ql = quad_lane(sub);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); base < a.m; base += stride) {
        const uint64_t k = base + lane;
        const bool live = k < a.m;
        uint64_t q = live ? a.q[k] : 0, r = 0;
        const bool bad = q > a.n;
        if (bad) q = 0;
        for (uint64_t t = 0; t < steps; t++) {
            r = rank_line_one<QUAD>(a, bl, ql, sub, q, a.c);
            if (t + 1 < steps) q = chain_next(q, r, a.n);
        }
        if (live) {
            a.out[2 * k] = bad ? ~0ull : q;
            a.out[2 * k + 1] = bad ? ~0ull : r;
            if (bad) atomicOr(a.status, kStatusRange);
        }
    }
}

template <int KIND>
KernelFn pick_line(int k) {
    switch (k) {
        case 1: return rank_line_kernel<1, KIND>;
        case 2: return rank_line_kernel<2, KIND>;
        default: return nullptr;
    }
}

}  // namespace

ChainFn pick_chain_line(bool quad) { return quad ? rank_chain_line_kernel<true> : rank_chain_line_kernel<false>; }

KernelFn pick_line_kind(int kind, int k) {
    switch (kind) {
        case kBiScalar: return pick_line<kBiScalar>(k);
        case kBiVec: return pick_line<kBiVec>(k);
        case kQuadScalar: return pick_line<kQuadScalar>(k);
        case kQuadVec: return pick_line<kQuadVec>(k);
        case kQuad4: return pick_line<kQuad4>(k);
        case kQuadPrefix: return pick_line<kQuadPrefix>(k);
        default: return nullptr;
    }
}

}  // namespace qr
