// Shared host/device helpers of the CUDA path: error reporting, layout
// constants of BiRank16 / QuadRank16, exact division by the block sizes,
// cache-hinted loads and stores, and the in-line query arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>

#include "quadrank.h"

namespace qr {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define QR_CUDA_TRY(call)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::qr::cuda_fail(e_, #call);  \
    } while (0)

// ---------------------------------------------------------------- layout
// BiRank16 (paper Sec. 3): a 64-byte line = 16-bit delta + B = 496 data bits,
// S = 128 blocks per superblock, superblock offsets shifted right by 11,
// deltas point to data offset 240 (line bit 256, the middle of the line).
constexpr uint64_t kB2 = 496;
constexpr uint64_t kSuper2 = 128;
constexpr uint64_t kMid2 = 240;
constexpr int kShift2 = 11;
// QuadRank16 (paper Sec. 4): four 16-bit deltas + B4 = 224 chars, 256 blocks
// per superblock, offsets shifted right by 13, deltas point to data index 96
// (slot 128, the middle of the line); slot = data index + 32.
constexpr uint64_t kB4 = 224;
constexpr uint64_t kSuper4 = 256;
constexpr uint64_t kMid4 = 96;
constexpr int kShift4 = 13;

// Sector layout (QR_LAYOUT_SECTOR): each 32-byte half of a line is
// self-contained.  sigma 2 (the paper's BiRank16x2, Sec. 3.1): a half holds a
// 16-bit delta + 240 data bits, a block (line) B = 480 bits, the delta points
// to data offset 120 of its half (1/4 and 3/4 of the block).  sigma 4: a half
// holds four 16-bit deltas + 96 chars (transposed: ~low bits of chars 0..63,
// ~high bits of chars 0..63, then ~low | ~high << 32 of chars 64..95), a line
// holds 192 chars, the deltas point to char 48 of the half.
constexpr uint64_t kB2s = 480;
constexpr uint64_t kHalf2s = 240;
constexpr uint64_t kMid2s = 120;
constexpr uint64_t kB4s = 192;
constexpr uint64_t kHalf4s = 96;
constexpr uint64_t kMid4s = 48;

// 128-byte line layout (QR_LAYOUT_LINE128): one DRAM line fill per query,
// read by the four lanes of a quad in one instruction.  sigma 2: a 16-bit
// delta + 1008 data bits per line (data bit d at line bit 16 + d), 32 lines
// per superblock, the delta points to data offset 504 (line bit 520).
// sigma 4: word 0 = four 16-bit deltas, word 1 = ~low | ~high << 32 of chars
// 448..479, words 2+2g / 3+2g = ~low / ~high bits of chars 64g..64g+63 for
// g = 0..6; 480 chars per line, 64 lines per superblock, deltas to char 240.
constexpr uint64_t kB2L = 1008;
constexpr uint64_t kMid2L = 504;
constexpr uint64_t kSuper2L = 32;
constexpr uint64_t kB4L = 480;
constexpr uint64_t kMid4L = 240;
constexpr uint64_t kSuper4L = 64;

// 32-bit inline layouts (QR_LAYOUT_INLINE32, QR_LAYOUT_INLINE32X2; paper
// Sec. 3.1 BiRank32 and BiRank32x2, Sec. 4.1 QuadRank32).  A 32-bit value per
// line (per half-line for BiRank32x2, per symbol for QuadRank32) holds the
// rank at the line's middle minus the rank at the start of its L0 block of
// 2^22 lines; the L0 table keeps one 64-bit rank per block (four for sigma
// 4), a few KB even at n = 2^43.  The values stay below 2^22 * 480 < 2^31.
//   BiRank32:   word 0 low 32 bits = value, data bit d (d < 480) at line bit
//               32 + d, the value counts data bits before offset 240.
//   BiRank32x2: each 32-byte half h: low 32 bits = value, data bit d (d < 224)
//               of the half at half bit 32 + d, the value counts the data bits
//               before offset 112 of the half.
//   QuadRank32: word 0 = v0 | v1 << 32, word 1 = v2 | v3 << 32; words 2 + 2g
//               / 3 + 2g = ~low / ~high bits of chars 64g .. 64g + 63 (g < 3);
//               v_c counts symbol c among chars 0 .. 95 of the line.
constexpr uint64_t kB2w = 480;
constexpr uint64_t kMid2w = 240;
constexpr uint64_t kB2x = 448;
constexpr uint64_t kHalf2x = 224;
constexpr uint64_t kMid2x = 112;
constexpr uint64_t kB4w = 192;
constexpr uint64_t kMid4w = 96;
constexpr int kL0Shift = 22;
constexpr uint64_t kL0Lines = 1ull << kL0Shift;
// QuadRank24_8 (QR_LAYOUT_INLINE24_8; paper Sec. 4.1): the chars and groups
// of QuadRank32, and per symbol c one 32-bit word a_c | b_c << 24 in words 0
// and 1 (as QuadRank32's values): a_c (24 bits) = rank at the end of group 0
// (char 64 of the line) minus the line's L0 entry, b_c (8 bits, <= 128) = the
// count of c in groups 1 and 2 (chars 64 .. 191), so that rank at the end of
// group 2 (char 192) = a_c + b_c.  A query in group 0 or 2 counts back from
// the end of its group, one in group 1 forward from its start: at most 64
// chars.  The 24-bit values need L0 blocks of 2^16 lines (2^16 * 192 < 2^24).
constexpr int kL0Shift24 = 16;
constexpr uint64_t kL0Lines24 = 1ull << kL0Shift24;

// Status bits written by kernels (same values as the QR_E* status codes).
constexpr uint32_t kStatusRange = QR_ERANGE;
constexpr uint32_t kStatusBadSym = QR_EBADSYM;
constexpr uint32_t kStatusTimeout = QR_ETIMEOUT;

// ---------------------------------------------------------------- division
// floor(q / 496) and floor(q / 224) for q < 2^63 without a 64-bit divide:
// 496 = 16 * 31 and 224 = 32 * 7; x / d = mulhi(x, ceil(2^(64+s) / d)) >> s is
// exact while x * (d * M - 2^(64+s)) < 2^(64+s) (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994).  Here
// x < 2^59 and the error terms are 23 (d = 31, s = 4) and 6 (d = 7, s = 2).
constexpr uint64_t kMagic31 = 0x8421084210842109ull;  // ceil(2^68 / 31)
constexpr uint64_t kMagic7 = 0x924924924924924Aull;   // ceil(2^66 / 7)

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
__host__ __device__ __forceinline__ uint64_t div496(uint64_t q) { return mulhi64(q >> 4, kMagic31) >> 4; }
__host__ __device__ __forceinline__ uint64_t div224(uint64_t q) { return mulhi64(q >> 5, kMagic7) >> 2; }
// 480 = 32 * 15 and 192 = 64 * 3, same method (error terms 7 and 1).
constexpr uint64_t kMagic15 = 0x8888888888888889ull;  // ceil(2^67 / 15)
constexpr uint64_t kMagic3 = 0xAAAAAAAAAAAAAAABull;   // ceil(2^65 / 3)
__host__ __device__ __forceinline__ uint64_t div480(uint64_t q) { return mulhi64(q >> 5, kMagic15) >> 3; }
// 1008 = 16 * 63 (error term 55).
constexpr uint64_t kMagic63 = 0x8208208208208209ull;  // ceil(2^69 / 63)
__host__ __device__ __forceinline__ uint64_t div1008(uint64_t q) { return mulhi64(q >> 4, kMagic63) >> 5; }
__host__ __device__ __forceinline__ uint64_t div192(uint64_t q) { return mulhi64(q >> 6, kMagic3) >> 1; }
// 448 = 64 * 7 (the magic of div224, error term 6).
__host__ __device__ __forceinline__ uint64_t div448(uint64_t q) { return mulhi64(q >> 6, kMagic7) >> 2; }
// floor(q / 224) for q < 2^32 with one 32-bit high multiply: x = q >> 5 and
// M = ceil(2^32 / 7) = (2^32 + 3) / 7 give x M / 2^32 = x / 7 + 3x / (7 2^32),
// which floors to floor(x / 7) while 3x < 2^32 (here x < 2^27).
__device__ __forceinline__ uint32_t div224_32(uint32_t q) { return __umulhi(q >> 5, 0x24924925u); }

// ---------------------------------------------------------------- bit helpers
__host__ __device__ __forceinline__ uint64_t low_mask(uint32_t nb) {  // nb in [0, 64]
    return nb >= 64 ? ~0ull : ((1ull << nb) - 1ull);
}
__host__ __device__ __forceinline__ uint32_t clamp64(int32_t v) {
    return (uint32_t)(v < 0 ? 0 : (v > 64 ? 64 : v));
}
__device__ __forceinline__ uint32_t popc64(uint64_t x) { return (uint32_t)__popcll(x); }
// Masks of 32-bit words.  low32(s) = the low s bits, s clamped to [0, 32]: the
// clamping funnel shift stops at 32 and max() handles s < 0.  cmask32 is the
// same for a compile-time s.  A range [X, M) or [M, X) with a fixed end M is
// low(X) XOR low(M), one funnel shift per word instead of two masks.
__device__ __forceinline__ uint32_t low32(int32_t s) {
    return __funnelshift_lc(0xFFFFFFFFu, 0u, (uint32_t)max(s, 0));
}
__host__ __device__ constexpr uint32_t cmask32(int s) { return s <= 0 ? 0u : s >= 32 ? ~0u : (1u << s) - 1u; }
__host__ __device__ __forceinline__ uint32_t lo32(uint64_t x) { return (uint32_t)x; }
__host__ __device__ __forceinline__ uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }

// ---------------------------------------------------------------- memory
// 16-byte loads of index lines: read-only path, no L1 allocation (a random
// line is touched once per query).
__device__ __forceinline__ uint4 ld_line16(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
// Four 64-bit words of one 32-byte sector.
struct u64x4 {
    uint64_t a, b, c, d;
};

// L2 cache policies (createpolicy, sm_80+) and loads that carry them: an
// evict-last policy for an index that should stay L2-resident while other
// data streams through, an evict-first policy for data read once.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ld_line16_hint(const uint4* p, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ u64x4 ld_line32_hint(const uint4* p, uint64_t pol) {
    u64x4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b64 {%0,%1,%2,%3}, [%4], %5;"
                 : "=l"(v.a), "=l"(v.b), "=l"(v.c), "=l"(v.d)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_u32_hint(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint64_t ld_u64_hint(const uint64_t* p, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}
// Streaming loads/stores of the query and result arrays (touched once).
__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint8_t ld_stream_u8(const uint8_t* p) {
    uint16_t v;
    asm volatile("ld.global.cs.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint8_t)v;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint16_t ld_stream_u16(const uint16_t* p) {
    uint16_t v;
    asm volatile("ld.global.cs.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_stream_v4u32(uint32_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint2 ld_stream_v2u32(const uint32_t* p) {
    uint2 v;
    asm volatile("ld.global.cs.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_stream_v4u32(const uint32_t* p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream_v2u64(uint64_t* p, uint64_t a, uint64_t b) {
    asm volatile("st.global.cs.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
// One 32-byte store (sm_100+ 256-bit vector store): a whole L2 sector written
// by one request, so the L2 needs no fill from DRAM.  p must be 32-byte aligned.
__device__ __forceinline__ void st_stream_v4u64(uint64_t* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    asm volatile("st.global.cs.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}
__device__ __forceinline__ void st_stream_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.global.cs.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 32-byte loads (sm_100+ 256-bit vector load): one instruction per sector.
__device__ __forceinline__ u64x4 ld_line32(const uint4* p) {
    u64x4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.b64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(v.a), "=l"(v.b), "=l"(v.c), "=l"(v.d)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ uint64_t lo64(uint4 v) { return (uint64_t)v.x | ((uint64_t)v.y << 32); }
__device__ __forceinline__ uint64_t hi64(uint4 v) { return (uint64_t)v.z | ((uint64_t)v.w << 32); }

// ---------------------------------------------------------------- BiRank16 query
// A line is 8 words w0..w7; bits 0..15 of w0 hold b_j, line bit 16 + d holds
// data bit jB + d (d < 496).  For p = q - jB:
//   p >= 240: rank = 2^11 s + b + popcount(line bits [256, 16 + p))
//   p <  240: rank = 2^11 s + b - popcount(line bits [16 + p, 256))
// (paper Sec. 3, Eq. 1).  `x` holds the four words of the half the query
// needs: w4..w7 when p >= 240, w0..w3 otherwise.
__device__ __forceinline__ uint64_t birank_finish(uint64_t s, uint64_t w0, const uint64_t x[4], uint32_t p) {
    const bool upper = p >= kMid2;
    // number of counted bits measured from the start of the selected half
    const int32_t t = upper ? (int32_t)(p - kMid2) : (int32_t)(16 + p);
    const uint32_t flip = upper ? 0u : ~0u;  // lower half: the bits at and above t
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
        cnt += __popc(lo32(x[k]) & (low32(t - 64 * k) ^ flip)) + __popc(hi32(x[k]) & (low32(t - 64 * k - 32) ^ flip));
    const uint64_t mid = (s << kShift2) + (w0 & 0xFFFFull);
    return upper ? mid + cnt : mid - cnt;
}

// ---------------------------------------------------------------- QuadRank16 query
// Line words: for half h and group g, word 4h+2g = ~(low bits) and word
// 4h+2g+1 = ~(high bits) of slots 128h+64g .. +63; the low 32 bits of words 0
// and 1 hold b_{j,0} | b_{j,1} << 16 and b_{j,2} | b_{j,3} << 16.
// slot = q - 224 j + 32; slot >= 128 adds the count of slots [128, slot),
// otherwise the count of slots [slot, 128) is subtracted (paper Sec. 4 and the
// rank1 listing of App. A).  x[0..3] = the 4 words of the needed half.
__device__ __forceinline__ uint64_t quad_delta(uint64_t w0, uint64_t w1, int c) {
    uint64_t w = (c & 2) ? w1 : w0;
    return (w >> (16 * (c & 1))) & 0xFFFFull;
}
// Slots 32 i .. 32 i + 31 of the needed half (i = 0..3) are the low (i even)
// or high (i odd) 32 bits of words x[2 (i / 2)] (~low bits) and x[2 (i / 2) + 1]
// (~high bits); m = the counted slots among them.
struct QuadHalf32 {
    uint32_t nl[4], nh[4], m[4];
};
__device__ __forceinline__ QuadHalf32 quad_half32(const uint64_t x[4], uint32_t slot) {
    const bool upper = slot >= 128;
    const int32_t t = upper ? (int32_t)(slot - 128) : (int32_t)slot;
    const uint32_t flip = upper ? 0u : ~0u;
    QuadHalf32 h;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint64_t L = x[2 * (i >> 1)], H = x[2 * (i >> 1) + 1];
        h.nl[i] = (i & 1) ? hi32(L) : lo32(L);
        h.nh[i] = (i & 1) ? hi32(H) : lo32(H);
        h.m[i] = low32(t - 32 * i) ^ flip;
    }
    return h;
}
__device__ __forceinline__ uint64_t quad_finish1(uint64_t s_c, uint64_t delta, const uint64_t x[4], uint32_t slot,
                                                 int c) {
    const QuadHalf32 h = quad_half32(x, slot);
    const uint32_t cl = 0u - (uint32_t)(c & 1), ch = 0u - (uint32_t)(c >> 1);
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) cnt += __popc((h.nl[i] ^ cl) & (h.nh[i] ^ ch) & h.m[i]);
    const uint64_t mid = (s_c << kShift4) + delta;
    return slot >= 128 ? mid + cnt : mid - cnt;
}
// All four counts of the masked slots: n3 = |L & H|, n1 = |L| - n3,
// n2 = |H| - n3, n0 = |mask| - n1 - n2 - n3 (L, H = raw low/high bits).
__device__ __forceinline__ void quad_finish4(const uint32_t s[4], uint64_t w0, uint64_t w1, const uint64_t x[4],
                                             uint32_t slot, uint64_t r[4]) {
    const QuadHalf32 h = quad_half32(x, slot);
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
    uint32_t n[4] = {nm - nl - nh + n3, nl - n3, nh - n3, n3};
#pragma unroll
    for (int c = 0; c < 4; c++) {
        uint64_t mid = ((uint64_t)s[c] << kShift4) + quad_delta(w0, w1, c);
        r[c] = upper ? mid + n[c] : mid - n[c];
    }
}

// ---------------------------------------------------------------- sector layout queries
// BiRank16x2 half-line: W = the 4 words of the query's 32-byte half, r = data
// offset inside the half (0..239).  Data offset d sits at half bit 16 + d; the
// delta counts the ones before data offset 120 of the half (half bit 136).
// Counted bits: low(16 + r) XOR low(136); the 16 delta bits lie under both.
__device__ __forceinline__ uint64_t birank_sector_finish(uint64_t s, const u64x4& W, uint32_t r) {
    const int32_t x = 16 + (int32_t)r;
    constexpr int kM = 16 + (int)kMid2s;
    const uint32_t w[8] = {lo32(W.a), hi32(W.a), lo32(W.b), hi32(W.b), lo32(W.c), hi32(W.c), lo32(W.d), hi32(W.d)};
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) cnt += __popc(w[i] & (low32(x - 32 * i) ^ cmask32(kM - 32 * i)));
    const uint64_t mid = (s << kShift2) + (W.a & 0xFFFFull);
    return r >= kMid2s ? mid + cnt : mid - cnt;
}
// QuadRank sector half: chars 0..31 and 32..63 are the low and high 32 bits
// of W.b (~low bits) and W.c (~high bits), chars 64..95 the low (~low bits)
// and high (~high bits) 32 bits of W.d; the deltas count chars before char 48.
struct QuadSector32 {
    uint32_t nl[3], nh[3], m[3];
};
__device__ __forceinline__ QuadSector32 quad_sector32(const u64x4& W, uint32_t r) {
    QuadSector32 h;
    h.nl[0] = lo32(W.b); h.nh[0] = lo32(W.c);
    h.nl[1] = hi32(W.b); h.nh[1] = hi32(W.c);
    h.nl[2] = lo32(W.d); h.nh[2] = hi32(W.d);
#pragma unroll
    for (int i = 0; i < 3; i++) h.m[i] = low32((int32_t)r - 32 * i) ^ cmask32((int)kMid4s - 32 * i);
    return h;
}
__device__ __forceinline__ uint64_t quad_sector_finish1(uint64_t s_c, const u64x4& W, uint32_t r, int c) {
    const QuadSector32 h = quad_sector32(W, r);
    const uint32_t cl = 0u - (uint32_t)(c & 1), ch = 0u - (uint32_t)(c >> 1);
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) cnt += __popc((h.nl[i] ^ cl) & (h.nh[i] ^ ch) & h.m[i]);
    const uint64_t mid = (s_c << kShift4) + ((W.a >> (16 * c)) & 0xFFFFull);
    return r >= kMid4s ? mid + cnt : mid - cnt;
}
__device__ __forceinline__ void quad_sector_finish4(const uint32_t s[4], const u64x4& W, uint32_t r, uint64_t out[4]) {
    const QuadSector32 h = quad_sector32(W, r);
    uint32_t nl = 0, nh = 0, n3 = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const uint32_t L = ~h.nl[i] & h.m[i], H = ~h.nh[i] & h.m[i];
        nl += __popc(L);
        nh += __popc(H);
        n3 += __popc(L & H);
    }
    const bool upper = r >= kMid4s;
    const uint32_t nm = upper ? r - (uint32_t)kMid4s : (uint32_t)kMid4s - r;
    const uint32_t n[4] = {nm - nl - nh + n3, nl - n3, nh - n3, n3};
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint64_t mid = ((uint64_t)s[c] << kShift4) + ((W.a >> (16 * c)) & 0xFFFFull);
        out[c] = upper ? mid + n[c] : mid - n[c];
    }
}

// ---------------------------------------------------------------- 32-bit inline layout queries
// A count over 32-bit words w[lo..hi) of the bits between bit position x and
// the fixed middle M (both measured in the words' bit coordinates): the mask
// of word i is low(x - 32 i) XOR low(M - 32 i).
template <int N, int FIRST, int M>
__device__ __forceinline__ uint32_t count_to_mid(const uint32_t (&w)[N], int32_t x) {
    uint32_t cnt = 0;
#pragma unroll
    for (int i = FIRST; i < N; i++) cnt += __popc(w[i] & (low32(x - 32 * i) ^ cmask32(M - 32 * i)));
    return cnt;
}
// BiRank32: the line's two sectors S0, S1, data offset d (< 480); l0 = the
// rank at the start of the line's L0 block.
__device__ __forceinline__ uint64_t in32_bi_finish(uint64_t l0, const u64x4& S0, const u64x4& S1, uint32_t d) {
    const uint32_t w[16] = {lo32(S0.a), hi32(S0.a), lo32(S0.b), hi32(S0.b), lo32(S0.c), hi32(S0.c),
                            lo32(S0.d), hi32(S0.d), lo32(S1.a), hi32(S1.a), lo32(S1.b), hi32(S1.b),
                            lo32(S1.c), hi32(S1.c), lo32(S1.d), hi32(S1.d)};
    const uint32_t cnt = count_to_mid<16, 1, 32 + (int)kMid2w>(w, 32 + (int32_t)d);
    const uint64_t mid = l0 + lo32(S0.a);
    return d >= kMid2w ? mid + cnt : mid - cnt;
}
// BiRank32x2: the query's 32-byte half W, data offset r inside the half (< 224).
__device__ __forceinline__ uint64_t in32x2_finish(uint64_t l0, const u64x4& W, uint32_t r) {
    const uint32_t w[8] = {lo32(W.a), hi32(W.a), lo32(W.b), hi32(W.b), lo32(W.c), hi32(W.c), lo32(W.d), hi32(W.d)};
    const uint32_t cnt = count_to_mid<8, 1, 32 + (int)kMid2x>(w, 32 + (int32_t)r);
    const uint64_t mid = l0 + lo32(W.a);
    return r >= kMid2x ? mid + cnt : mid - cnt;
}
// QuadRank32: chars 32 i .. 32 i + 31 (i < 6) are the low (i even) or high
// (i odd) 32 bits of words 2 + 2 (i / 2) (~low bits) and 3 + 2 (i / 2)
// (~high bits); the mask of each is the chars between d and 96.
struct Quad32Words {
    uint32_t nl[6], nh[6], m[6];
};
__device__ __forceinline__ Quad32Words quad32_words(const u64x4& S0, const u64x4& S1, uint32_t d) {
    const uint64_t L[3] = {S0.c, S1.a, S1.c}, H[3] = {S0.d, S1.b, S1.d};
    Quad32Words q;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        q.nl[i] = (i & 1) ? hi32(L[i >> 1]) : lo32(L[i >> 1]);
        q.nh[i] = (i & 1) ? hi32(H[i >> 1]) : lo32(H[i >> 1]);
        q.m[i] = low32((int32_t)d - 32 * i) ^ cmask32((int)kMid4w - 32 * i);
    }
    return q;
}
__device__ __forceinline__ uint32_t quad32_value(const u64x4& S0, int c) {
    const uint64_t w = (c & 2) ? S0.b : S0.a;
    return (c & 1) ? hi32(w) : lo32(w);
}
__device__ __forceinline__ uint64_t quad32_finish1(uint64_t l0_c, const u64x4& S0, const u64x4& S1, uint32_t d,
                                                   int c) {
    const Quad32Words q = quad32_words(S0, S1, d);
    const uint32_t cl = 0u - (uint32_t)(c & 1), ch = 0u - (uint32_t)(c >> 1);
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 6; i++) cnt += __popc((q.nl[i] ^ cl) & (q.nh[i] ^ ch) & q.m[i]);
    const uint64_t mid = l0_c + quad32_value(S0, c);
    return d >= kMid4w ? mid + cnt : mid - cnt;
}
// All four counts: n3 = |L & H|, n1 = |L| - n3, n2 = |H| - n3,
// n0 = |mask| - n1 - n2 - n3 over the masked chars (L, H = raw bits).
__device__ __forceinline__ void quad32_finish4(const uint64_t l0[4], const u64x4& S0, const u64x4& S1, uint32_t d,
                                               uint64_t r[4]) {
    const Quad32Words q = quad32_words(S0, S1, d);
    uint32_t nl = 0, nh = 0, n3 = 0;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const uint32_t L = ~q.nl[i] & q.m[i], H = ~q.nh[i] & q.m[i];
        nl += __popc(L);
        nh += __popc(H);
        n3 += __popc(L & H);
    }
    const bool upper = d >= kMid4w;
    const uint32_t nm = upper ? d - (uint32_t)kMid4w : (uint32_t)kMid4w - d;
    const uint32_t n[4] = {nm - nl - nh + n3, nl - n3, nh - n3, n3};
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint64_t mid = l0[c] + quad32_value(S0, c);
        r[c] = upper ? mid + n[c] : mid - n[c];
    }
}

// QuadRank24_8: position d (< 192) of a line whose sectors are S0, S1.  The
// group g = d / 64 holds the counted chars: [d, 64 g + 64) subtracted from
// the rank at the group's end for g = 0 and 2, [64, d) added to the rank at
// char 64 for g = 1.
struct Quad24Words {
    uint64_t nl, nh, m;  // the group's ~low / ~high words and the mask of the counted chars
    uint32_t g;
};
__device__ __forceinline__ Quad24Words quad24_words(const u64x4& S0, const u64x4& S1, uint32_t d) {
    Quad24Words q;
    q.g = d >> 6;
    const uint32_t t = d & 63;
    q.nl = q.g == 0 ? S0.c : q.g == 1 ? S1.a : S1.c;
    q.nh = q.g == 0 ? S0.d : q.g == 1 ? S1.b : S1.d;
    const uint64_t below = low_mask(t);  // chars 64 g .. 64 g + t - 1
    q.m = q.g == 1 ? below : ~below;
    return q;
}
// The rank at the reference point of group g for symbol c: l0 + a_c, plus b_c
// for group 2.
__device__ __forceinline__ uint64_t quad24_mid(uint64_t l0_c, const u64x4& S0, int c, uint32_t g) {
    const uint32_t v = quad32_value(S0, c);
    return l0_c + (v & 0xFFFFFFu) + (g == 2 ? (v >> 24) : 0u);
}
__device__ __forceinline__ uint64_t quad24_finish1(uint64_t l0_c, const u64x4& S0, const u64x4& S1, uint32_t d,
                                                   int c) {
    const Quad24Words q = quad24_words(S0, S1, d);
    const uint64_t cl = 0ull - (uint64_t)(c & 1), ch = 0ull - (uint64_t)(c >> 1);
    const uint32_t cnt = popc64((q.nl ^ cl) & (q.nh ^ ch) & q.m);
    const uint64_t mid = quad24_mid(l0_c, S0, c, q.g);
    return q.g == 1 ? mid + cnt : mid - cnt;
}
__device__ __forceinline__ void quad24_finish4(const uint64_t l0[4], const u64x4& S0, const u64x4& S1, uint32_t d,
                                               uint64_t r[4]) {
    const Quad24Words q = quad24_words(S0, S1, d);
    const uint64_t L = ~q.nl & q.m, H = ~q.nh & q.m;
    const uint32_t n3 = popc64(L & H), nl = popc64(L), nh = popc64(H), nm = popc64(q.m);
    const uint32_t n[4] = {nm - nl - nh + n3, nl - n3, nh - n3, n3};
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint64_t mid = quad24_mid(l0[c], S0, c, q.g);
        r[c] = q.g == 1 ? mid + n[c] : mid - n[c];
    }
}

// ---------------------------------------------------------------- host side
struct DeviceProps {
    int device = -1;
    int sms = 0;
    int l2_bytes = 0;
};
const DeviceProps& device_props();

}  // namespace qr

// Opaque handle of a rank index (see quadrank.h).
struct qr_index {
    int sigma = 2;
    int layout = QR_LAYOUT_PAPER;
    uint64_t n = 0;
    uint64_t nblocks = 0, nsuper = 0;
    uint4* lines = nullptr;      // nblocks x 64 B
    void* supers = nullptr;      // sigma 2: uint32[nsuper]; sigma 4: uint4[nsuper]
    uint32_t* status = nullptr;  // device status word
    int device = 0;
    qr_tuning_t tune{4, 256, 0, 0};
    int batch_mode = QR_BATCH_AUTO;  // direct kernels or region batching (qr_set_batch_mode)
    int region_variant = 0;          // rank pass launch variant, 0..3 (qr_set_region_tuning)
    bool region_timing = false;      // record events between the region passes
    int region_withhold = 0;         // test hook (qr_set_region_fault)
    cudaEvent_t region_ev[4] = {};
    // host-buffer pipeline (lazy): kPipe streams, one staging slot each
    static constexpr int kPipe = 4;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t pipe[kPipe] = {};
    cudaEvent_t ev[kPipe + 1] = {};
};

namespace qr {
uint64_t block_chars(int sigma, int layout);
uint64_t super_lines(int sigma, int layout);
uint64_t line_bytes(int layout);
uint64_t super_entry_bytes(int sigma, int layout);
inline bool inline_layout(int layout) {
    return layout == QR_LAYOUT_INLINE32 || layout == QR_LAYOUT_INLINE32X2 || layout == QR_LAYOUT_INLINE24_8;
}
// log2 of the lines per L0 entry of an inline layout
inline int l0_shift(int layout) { return layout == QR_LAYOUT_INLINE24_8 ? kL0Shift24 : kL0Shift; }
// Build the layout into an already sized index from a device text.
int build_rank_index(qr_index* idx, const uint64_t* d_text, cudaStream_t s);
// Launch the rank kernels (no argument checks beyond the mode); rank4 = 0:
// rank(q, c), 1: rank_4, 2: prefix_rank(q, c).
int launch_rank(const qr_index* idx, const uint64_t* q, const uint8_t* cvec, int c, uint64_t m, uint64_t* out,
                int rank4, cudaStream_t s);
// The direct kernels alone (gate: see RankArgs; NULL = always run).
int launch_direct(const qr_index* idx, const uint64_t* q, const uint8_t* cvec, int c, uint64_t m, uint64_t* out,
                  int rank4, cudaStream_t s, const unsigned long long* gate, unsigned long long gate_limit);
int launch_chain(const qr_index* idx, const uint64_t* q0, uint64_t nchains, uint64_t steps, int c, uint64_t* out,
                 cudaStream_t s);
// Region batching (qr_region.cu): which calls it serves, the automatic rule,
// the launch (marks: 4 events recorded around the three passes, or NULL) and
// the release of its pooled scratch.
bool region_supported(const qr_index* idx, int rank4);
bool region_auto(const qr_index* idx, uint64_t m);
// direct (may be NULL): launches the direct kernels gated by a device count
// (they run only when *count <= limit); with it, region batching adds the
// probe that sets the count, and its passes run only when *count > limit.
using DirectLaunch = std::function<int(const unsigned long long* count, unsigned long long limit)>;
int launch_rank_regions(const qr_index* idx, const uint64_t* q, const uint8_t* cvec, int c, uint64_t m, uint64_t* out,
                        int rank4, cudaStream_t s, cudaEvent_t* marks, const DirectLaunch* direct);
int region_trim();
int launch_probe(const void* buf, uint64_t nrec, int bytes, int load_bytes, uint64_t m, uint64_t seed, uint64_t* out,
                 int k, int threads, cudaStream_t s);
int launch_probe_l2(const void* buf, uint64_t nrec, int mode, uint64_t nthreads, uint32_t rounds, uint64_t seed,
                    uint64_t* out, int threads, cudaStream_t s);
}  // namespace qr
