// QuadFm index handle and the rank step of the backward search, shared by the
// builder and the count kernels.
#pragma once

#include "qr_common.cuh"

constexpr int kQfmK = 8;                  // prefix-table length (paper App. D)
constexpr uint64_t kQfmTable = 1ull << 16; // 4^8 entries

// Opaque handle of a count-only FM-index (see quadfm.h).
struct qfm_index {
    uint64_t n = 0;            // text length; the BWT has n + 1 rows
    uint64_t dollar_row = 0;   // BWT row of $ (stored as code 0 in the rank index)
    uint64_t C[5] = {0, 0, 0, 0, 0};
    qr_index* rank = nullptr;  // QuadRank16 over the BWT
    uint64_t* table = nullptr; // [4^8][2] : [lo, hi) of every 8-mer
    uint32_t* sa = nullptr;    // suffix array (only with QFM_KEEP_SA)
    uint32_t* status = nullptr;
    int device = 0;
    int policy = 2;            // kFmPolicy* of the persistent count kernel
    // locate (built when a sampling factor is given): rows whose suffix
    // starts at a multiple of sa_sample are marked in a BiRank16 index over
    // the n + 1 rows; samples[rank1(marks, row)] = SA[row] / sa_sample.
    uint32_t sa_sample = 0;
    qr_index* marks = nullptr;
    uint32_t* samples = nullptr;
    uint64_t nsamples = 0;
};

namespace qr {

// Everything a search step needs, passed by value to the kernels.
struct FmView {
    const uint4* __restrict__ lines;
    const uint4* __restrict__ supers;  // 4 x uint32 per superblock
    const uint64_t* __restrict__ table;
    uint64_t nrows;                    // n + 1
    uint64_t dollar;
    uint64_t C[4];
};

// L2 policies of the persistent count kernel (qfm_index::policy).
constexpr int kFmPolicyDefault = 0;   // read-only path, no L1 allocation
constexpr int kFmPolicyKeepIndex = 1; // index evict-last, patterns/offsets evict-first
constexpr int kFmPolicyKeepIndexOnly = 2; // index evict-last, patterns/offsets the default L2 policy

// 16-byte index load with the chosen L2 policy (KEEP: the evict-last policy `pol`).
template <bool KEEP>
__device__ __forceinline__ uint4 fm_ld(const uint4* p, uint64_t pol) {
    return KEEP ? ld_line16_hint(p, pol) : ld_line16(p);
}

// rank(q, c) over the BWT with the sentinel row counted as code 0.
template <bool KEEP = false>
__device__ __forceinline__ uint64_t fm_rank_stored(const FmView& v, uint64_t q, int c, uint64_t pol = 0) {
    const uint64_t j = div224_32((uint32_t)q);  // BWT rows < 2^32
    const uint32_t slot = (uint32_t)(q - j * kB4) + 32;
    const uint4* L = v.lines + 4 * j;
    const uint32_t* sp = (const uint32_t*)v.supers + 4 * (j >> 8) + c;
    const uint32_t s = KEEP ? ld_u32_hint(sp, pol) : __ldg(sp);
    const uint4 v0 = fm_ld<KEEP>(L, pol);
    const bool upper = slot >= 128;
    const uint4 va = fm_ld<KEEP>(L + (upper ? 2 : 1), pol);
    uint64_t x[4];
    if (upper) {
        const uint4 vb = fm_ld<KEEP>(L + 3, pol);
        x[0] = lo64(va); x[1] = hi64(va); x[2] = lo64(vb); x[3] = hi64(vb);
    } else {
        x[0] = lo64(v0); x[1] = hi64(v0); x[2] = lo64(va); x[3] = hi64(va);
    }
    return quad_finish1(s, quad_delta(lo64(v0), hi64(v0), c), x, slot, c);
}

// The words one rank query needs from its line, fetched as 32-byte sectors:
// sector 0 (deltas + the lower half) for slots below 128; the first 16 bytes
// (deltas) and sector 1 for the upper half.
struct FmLine {
    uint64_t d0, d1;     // words 0 and 1 (deltas in their low 32 bits)
    uint64_t x[4];       // the 4 words of the needed half
};

template <bool KEEP>
__device__ __forceinline__ FmLine fm_fetch(const uint4* L, bool upper, uint64_t pol) {
    FmLine f;
    if (upper) {
        const uint4 v0 = KEEP ? ld_line16_hint(L, pol) : ld_line16(L);
        const u64x4 s1 = KEEP ? ld_line32_hint(L + 2, pol) : ld_line32(L + 2);
        f.d0 = lo64(v0); f.d1 = hi64(v0);
        f.x[0] = s1.a; f.x[1] = s1.b; f.x[2] = s1.c; f.x[3] = s1.d;
    } else {
        const u64x4 s0 = KEEP ? ld_line32_hint(L, pol) : ld_line32(L);
        f.d0 = s0.a; f.d1 = s0.b;
        f.x[0] = s0.a; f.x[1] = s0.b; f.x[2] = s0.c; f.x[3] = s0.d;
    }
    return f;
}

// C[c] by selects: indexing the kernel-parameter array with a run-time c
// would copy the whole argument block to local memory.
__device__ __forceinline__ uint64_t fm_C(const FmView& v, int c) {
    return c == 0 ? v.C[0] : c == 1 ? v.C[1] : c == 2 ? v.C[2] : v.C[3];
}

// rank(q, c) of one interval end from its fetched words, in 32-bit
// arithmetic (BWT rows < 2^32): 2^13 s + delta +- the masked count.
__device__ __forceinline__ uint32_t fm_finish32(uint32_t s, const FmLine& f, uint32_t slot, int c) {
    const uint32_t dw = (c & 2) ? lo32(f.d1) : lo32(f.d0);
    const uint32_t delta = (dw >> (16 * (c & 1))) & 0xFFFFu;
    const QuadHalf32 h = quad_half32(f.x, slot);
    const uint32_t cl = 0u - (uint32_t)(c & 1), ch = 0u - (uint32_t)(c >> 1);
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) cnt += __popc((h.nl[i] ^ cl) & (h.nh[i] ^ ch) & h.m[i]);
    const uint32_t mid = (s << kShift4) + delta;
    return slot >= 128 ? mid + cnt : mid - cnt;
}

// LF of both interval ends for symbol c.  When lo and hi fall in the same
// half-line (the interval is narrow, the usual case after a few steps) the
// words are fetched once.  The $ row (stored as code 0) is removed from the
// count of c = 0 when it lies before the position.
template <bool KEEP>
__device__ __forceinline__ void fm_lf_pair(const FmView& v, uint32_t& lo, uint32_t& hi, int c, uint64_t pol) {
    const uint32_t jl = div224_32(lo), jh = div224_32(hi);
    const uint32_t sl = lo - jl * (uint32_t)kB4 + 32, sh = hi - jh * (uint32_t)kB4 + 32;
    const bool ul = sl >= 128, uh = sh >= 128;
    const uint32_t* sp = (const uint32_t*)v.supers + c;
    const uint32_t s_lo = KEEP ? ld_u32_hint(sp + 4 * (jl >> 8), pol) : __ldg(sp + 4 * (jl >> 8));
    const uint32_t s_hi = jl >> 8 == jh >> 8 ? s_lo : (KEEP ? ld_u32_hint(sp + 4 * (jh >> 8), pol) : __ldg(sp + 4 * (jh >> 8)));
    const FmLine fl = fm_fetch<KEEP>(v.lines + 4 * (uint64_t)jl, ul, pol);
    const FmLine fh = (jl == jh && ul == uh) ? fl : fm_fetch<KEEP>(v.lines + 4 * (uint64_t)jh, uh, pol);
    uint32_t rl = fm_finish32(s_lo, fl, sl, c);
    uint32_t rh = fm_finish32(s_hi, fh, sh, c);
    if (c == 0) {
        const uint32_t d = (uint32_t)v.dollar;
        rl -= lo > d ? 1u : 0u;
        rh -= hi > d ? 1u : 0u;
    }
    const uint32_t Cc = (uint32_t)fm_C(v, c);
    lo = Cc + rl;
    hi = Cc + rh;
}

// LF step of one interval end: C[c] + rank(q, c), where the $ row (stored as
// code 0) is removed from the count of c = 0 when it lies before q.
template <bool KEEP = false>
__device__ __forceinline__ uint64_t fm_lf(const FmView& v, uint64_t q, int c, uint64_t pol = 0) {
    uint64_t r = fm_rank_stored<KEEP>(v, q, c, pol);
    if (c == 0 && q > v.dollar) r -= 1;
    return fm_C(v, c) + r;
}

// BWT char of row r and LF(r) = C[c] + rank(r, c) - [c = 0 and r > dollar],
// both from the half-line that holds r (its slot lies in the counted half).
// The $ row is never passed (it is marked for locate: its suffix starts at 0).
__device__ __forceinline__ uint32_t fm_lf_row(const FmView& v, uint32_t r) {
    const uint32_t j = div224_32(r);
    const uint32_t slot = r - j * (uint32_t)kB4 + 32;
    const bool upper = slot >= 128;
    const uint4 s4 = __ldg(v.supers + (j >> 8));
    const FmLine f = fm_fetch<false>(v.lines + 4 * (uint64_t)j, upper, 0);
    const uint32_t t = slot - (upper ? 128u : 0u), g = t >> 6, b = t & 63;
    const uint64_t nl = g ? f.x[2] : f.x[0], nh = g ? f.x[3] : f.x[1];
    const int c = (int)(((~nl >> b) & 1) | (((~nh >> b) & 1) << 1));
    const uint32_t sc = c == 0 ? s4.x : c == 1 ? s4.y : c == 2 ? s4.z : s4.w;
    uint32_t rk = fm_finish32(sc, f, slot, c);
    if (c == 0 && r > (uint32_t)v.dollar) rk -= 1;
    return (uint32_t)fm_C(v, c) + rk;
}

// rank1(q) over a BiRank16 index in the paper layout (64-byte lines).
__device__ __forceinline__ uint64_t birank_rank_paper(const uint4* __restrict__ lines, const uint32_t* __restrict__ supers,
                                                      uint64_t q) {
    const uint64_t j = div496(q);
    const uint32_t p = (uint32_t)(q - j * kB2);
    const bool upper = p >= kMid2;
    const uint4* L = lines + 4 * j;
    const u64x4 S = ld_line32(L + (upper ? 2 : 0));
    const uint64_t w0 = upper ? __ldg((const unsigned long long*)L) : S.a;
    const uint64_t x[4] = {S.a, S.b, S.c, S.d};
    return birank_finish(__ldg(supers + (j >> 7)), w0, x, p);
}

// Bit q of the bit string held in a BiRank16 paper-layout index.
__device__ __forceinline__ bool birank_bit_paper(const uint4* __restrict__ lines, uint64_t q) {
    const uint64_t j = div496(q);
    const uint32_t b = (uint32_t)(q - j * kB2) + 16;  // line bit of data offset q - jB
    const uint64_t w = __ldg((const unsigned long long*)lines + 8 * j + (b >> 6));
    return (w >> (b & 63)) & 1;
}

int fm_view(const qfm_index* idx, FmView* v);

// The persistent count launch (qfm_count.cu): counts of m patterns (2 m with
// strands = 2) into out; with lohi, also each search's final interval.
int launch_count(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                 unsigned long long* queue, cudaStream_t s, int strands, uint64_t* lohi = nullptr);

}  // namespace qr
