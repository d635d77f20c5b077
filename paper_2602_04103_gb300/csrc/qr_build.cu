// Layout builder of BiRank16 and QuadRank16 (paper Sec. 3 "Parallel
// construction" and Sec. 4): one warp per superblock counts its blocks, an
// exclusive scan turns superblock counts into absolute ranks, and a second
// pass writes every 64-byte line (deltas to the block middle + data) and the
// shifted superblock offsets.
#include <cuda_runtime.h>

#include "qr_common.cuh"
#include "qr_scan.cuh"

namespace qr {
namespace {

constexpr int kWarpsPerBlock = 8;

// 64 bits of a packed bit stream starting at bit o; bits >= nbits are 0 and
// no word at or beyond ceil(nbits / 64) is read.
__device__ __forceinline__ uint64_t bits64(const uint64_t* __restrict__ t, uint64_t nbits, uint64_t o) {
    if (o >= nbits) return 0;
    const uint64_t w = o >> 6;
    const uint32_t sh = (uint32_t)(o & 63);
    const uint64_t nwords = (nbits + 63) >> 6;
    uint64_t v = t[w] >> sh;
    if (sh != 0 && w + 1 < nwords) v |= t[w + 1] << (64 - sh);
    const uint64_t left = nbits - o;
    if (left < 64) v &= low_mask((uint32_t)left);
    return v;
}

// ---------------------------------------------------------------- sigma = 2
// The 8 words of line j (b_j not yet inserted: word 0 holds data bits
// [jB, jB + 48) in bits 16..63) and the counts of the whole block and of its
// first 240 bits.
struct Line2 {
    uint64_t w[8];
    uint32_t cnt, half;
};

__device__ __forceinline__ Line2 make_line2(const uint64_t* __restrict__ t, uint64_t n, uint64_t j) {
    Line2 L;
    const uint64_t base = j * kB2;
    L.w[0] = bits64(t, n, base) << 16;
#pragma unroll
    for (int k = 1; k < 8; k++) L.w[k] = bits64(t, n, base + 64 * k - 16);
    uint32_t h = popc64(L.w[0]) + popc64(L.w[1]) + popc64(L.w[2]) + popc64(L.w[3]);
    L.half = h;
    L.cnt = h + popc64(L.w[4]) + popc64(L.w[5]) + popc64(L.w[6]) + popc64(L.w[7]);
    return L;
}

__global__ void count2_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                              uint64_t* __restrict__ super_cnt) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t sum = 0;
        for (int r = 0; r < (int)(kSuper2 / 32); r++) {
            uint64_t j = i * kSuper2 + r * 32 + lane;
            if (j < nblocks) sum += make_line2(text, n, j).cnt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) super_cnt[i] = sum;
    }
}

__global__ void layout2_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                               const uint64_t* __restrict__ super_base, uint4* __restrict__ lines,
                               uint32_t* __restrict__ supers) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        const uint64_t base = super_base[i];
        const uint64_t s = base >> kShift2;  // paper: s_i = floor(rank(iS) / 2^11)
        if (lane == 0) supers[i] = (uint32_t)s;
        uint64_t running = base - (s << kShift2);  // rank(iS) mod 2^11, folded into every b_j
        for (int r = 0; r < (int)(kSuper2 / 32); r++) {
            const uint64_t j = i * kSuper2 + r * 32 + lane;
            Line2 L;
            if (j < nblocks) L = make_line2(text, n, j);
            else L.cnt = 0, L.half = 0;
            uint32_t incl = L.cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint64_t before = running + (incl - L.cnt);  // rank(jB) - 2^11 s_i
            if (j < nblocks) {
                const uint64_t b = before + L.half;  // rank(jB + 240) - 2^11 s_i  < 2^16
                L.w[0] |= b;
                uint4* dst = lines + 4 * j;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    dst[k] = make_uint4((uint32_t)L.w[2 * k], (uint32_t)(L.w[2 * k] >> 32), (uint32_t)L.w[2 * k + 1],
                                        (uint32_t)(L.w[2 * k + 1] >> 32));
            }
            running += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// ---------------------------------------------------------------- sigma = 4
// Gather the low and high bits of 32 consecutive chars (one 64-bit window of
// the 2-bit packed text) into two 32-bit values.
__device__ __forceinline__ uint32_t even_bits(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}

struct Line4 {
    uint64_t w[8];     // final words except the delta bits of w0, w1
    uint32_t cnt[4];   // per-symbol count of the 224 chars
    uint32_t half[4];  // per-symbol count of the first 96 chars
};

__device__ __forceinline__ void count_group(uint64_t L, uint64_t H, uint64_t valid, uint32_t c[4]) {
    c[0] += popc64(~L & ~H & valid);
    c[1] += popc64(L & ~H & valid);
    c[2] += popc64(~L & H & valid);
    c[3] += popc64(L & H & valid);
}

__device__ __forceinline__ Line4 make_line4(const uint64_t* __restrict__ t, uint64_t n, uint64_t j) {
    Line4 R;
    const uint64_t nbits = 2 * n;
    const uint64_t c0 = j * kB4;  // first char of the block
    uint32_t cnt[4] = {0, 0, 0, 0};
    // group (0,0): slots 32..63 = chars c0 .. c0+31 (slots 0..31 carry the deltas)
    {
        uint64_t x = bits64(t, nbits, 2 * c0);
        uint64_t L = (uint64_t)even_bits(x) << 32, H = (uint64_t)even_bits(x >> 1) << 32;
        count_group(L, H, 0xFFFFFFFF00000000ull, cnt);
        R.w[0] = ~L;
        R.w[1] = ~H;
    }
    // groups (0,1), (1,0), (1,1): slots 64(1+g') .. +63 = chars c0 + 32 + 64 g' .. +63
#pragma unroll
    for (int gg = 0; gg < 3; gg++) {
        const uint64_t first = c0 + 32 + 64 * gg;
        uint64_t x0 = bits64(t, nbits, 2 * first), x1 = bits64(t, nbits, 2 * first + 64);
        uint64_t L = (uint64_t)even_bits(x0) | ((uint64_t)even_bits(x1) << 32);
        uint64_t H = (uint64_t)even_bits(x0 >> 1) | ((uint64_t)even_bits(x1 >> 1) << 32);
        if (gg == 0) {
#pragma unroll
            for (int c = 0; c < 4; c++) R.half[c] = cnt[c];
            count_group(L, H, ~0ull, R.half);
        }
        count_group(L, H, ~0ull, cnt);
        R.w[2 + 2 * gg] = ~L;
        R.w[3 + 2 * gg] = ~H;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) R.cnt[c] = cnt[c];
    return R;
}

__global__ void count4_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                              uint64_t* __restrict__ super_cnt /* [4][nsuper] */) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t sum[4] = {0, 0, 0, 0};
        for (int r = 0; r < (int)(kSuper4 / 32); r++) {
            uint64_t j = i * kSuper4 + r * 32 + lane;
            if (j < nblocks) {
                Line4 L = make_line4(text, n, j);
#pragma unroll
                for (int c = 0; c < 4; c++) sum[c] += L.cnt[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
            if (lane == 0) super_cnt[c * nsuper + i] = sum[c];
        }
    }
}

__global__ void layout4_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                               const uint64_t* __restrict__ super_base /* [4][nsuper] */, uint4* __restrict__ lines,
                               uint4* __restrict__ supers) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t running[4];
        uint32_t s[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint64_t base = super_base[c * nsuper + i];
            s[c] = (uint32_t)(base >> kShift4);  // paper: s_{i,c} = floor(rank(iS4, c) / 2^13)
            running[c] = base - ((uint64_t)s[c] << kShift4);
        }
        if (lane == 0) supers[i] = make_uint4(s[0], s[1], s[2], s[3]);
        for (int r = 0; r < (int)(kSuper4 / 32); r++) {
            const uint64_t j = i * kSuper4 + r * 32 + lane;
            Line4 L;
            const bool live = j < nblocks;
            if (live) L = make_line4(text, n, j);
            uint64_t b[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                uint32_t v = live ? L.cnt[c] : 0, incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                b[c] = running[c] + (incl - v) + (live ? L.half[c] : 0);  // rank(jB4 + 96, c) - 2^13 s_{i,c}
                running[c] += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (live) {
                L.w[0] = (L.w[0] & 0xFFFFFFFF00000000ull) | b[0] | (b[1] << 16);
                L.w[1] = (L.w[1] & 0xFFFFFFFF00000000ull) | b[2] | (b[3] << 16);
                uint4* dst = lines + 4 * j;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    dst[k] = make_uint4((uint32_t)L.w[2 * k], (uint32_t)(L.w[2 * k] >> 32), (uint32_t)L.w[2 * k + 1],
                                        (uint32_t)(L.w[2 * k + 1] >> 32));
            }
        }
    }
}

// ---------------------------------------------------------------- sector layout
// sigma 2 (BiRank16x2): half h of line j holds data bits [480j + 240h, +240)
// at half bits 16..255 and its delta in bits 0..15.
struct Half2 {
    uint64_t w[4];
    uint32_t cnt, quarter;  // ones in the 240 bits / in their first 120 bits
};

__device__ __forceinline__ Half2 make_half2(const uint64_t* __restrict__ t, uint64_t n, uint64_t base) {
    Half2 H;
    H.w[0] = bits64(t, n, base) << 16;
    H.w[1] = bits64(t, n, base + 48);
    H.w[2] = bits64(t, n, base + 112);
    H.w[3] = bits64(t, n, base + 176);
    H.quarter = popc64(H.w[0]) + popc64(H.w[1]) + popc64(H.w[2] & 0xFFull);
    H.cnt = popc64(H.w[0]) + popc64(H.w[1]) + popc64(H.w[2]) + popc64(H.w[3]);
    return H;
}

__global__ void count2s_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                               uint64_t* __restrict__ super_cnt) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t sum = 0;
        for (int r = 0; r < (int)(kSuper2 / 32); r++) {
            const uint64_t j = i * kSuper2 + r * 32 + lane;
            if (j < nblocks) sum += make_half2(text, n, j * kB2s).cnt + make_half2(text, n, j * kB2s + kHalf2s).cnt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) super_cnt[i] = sum;
    }
}

__global__ void layout2s_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                                const uint64_t* __restrict__ super_base, uint4* __restrict__ lines,
                                uint32_t* __restrict__ supers) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        const uint64_t base = super_base[i];
        const uint64_t s = base >> kShift2;
        if (lane == 0) supers[i] = (uint32_t)s;
        uint64_t running = base - (s << kShift2);
        for (int r = 0; r < (int)(kSuper2 / 32); r++) {
            const uint64_t j = i * kSuper2 + r * 32 + lane;
            const bool live = j < nblocks;
            Half2 h0, h1;
            if (live) {
                h0 = make_half2(text, n, j * kB2s);
                h1 = make_half2(text, n, j * kB2s + kHalf2s);
            }
            const uint32_t v = live ? h0.cnt + h1.cnt : 0;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (live) {
                const uint64_t before = running + (incl - v);  // rank(jB) - 2^11 s_i
                h0.w[0] |= before + h0.quarter;                // rank(jB + 120) - 2^11 s_i
                h1.w[0] |= before + h0.cnt + h1.quarter;       // rank(jB + 360) - 2^11 s_i
                uint4* dst = lines + 4 * j;
                dst[0] = make_uint4((uint32_t)h0.w[0], (uint32_t)(h0.w[0] >> 32), (uint32_t)h0.w[1],
                                    (uint32_t)(h0.w[1] >> 32));
                dst[1] = make_uint4((uint32_t)h0.w[2], (uint32_t)(h0.w[2] >> 32), (uint32_t)h0.w[3],
                                    (uint32_t)(h0.w[3] >> 32));
                dst[2] = make_uint4((uint32_t)h1.w[0], (uint32_t)(h1.w[0] >> 32), (uint32_t)h1.w[1],
                                    (uint32_t)(h1.w[1] >> 32));
                dst[3] = make_uint4((uint32_t)h1.w[2], (uint32_t)(h1.w[2] >> 32), (uint32_t)h1.w[3],
                                    (uint32_t)(h1.w[3] >> 32));
            }
            running += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// sigma 4 sector layout: half h of line j holds chars [192j + 96h, +96).
struct Half4 {
    uint64_t w[4];     // w[0] (deltas) left 0 here
    uint32_t cnt[4];   // per-symbol count of the 96 chars
    uint32_t mid[4];   // per-symbol count of the first 48 chars
};

__device__ __forceinline__ Half4 make_half4(const uint64_t* __restrict__ t, uint64_t n, uint64_t c0) {
    Half4 H;
    const uint64_t nbits = 2 * n;
    const uint64_t x0 = bits64(t, nbits, 2 * c0), x1 = bits64(t, nbits, 2 * c0 + 64), x2 = bits64(t, nbits, 2 * c0 + 128);
    const uint64_t LA = (uint64_t)even_bits(x0) | ((uint64_t)even_bits(x1) << 32);
    const uint64_t HA = (uint64_t)even_bits(x0 >> 1) | ((uint64_t)even_bits(x1 >> 1) << 32);
    const uint64_t LB = even_bits(x2), HB = even_bits(x2 >> 1);
    H.w[0] = 0;
    H.w[1] = ~LA;
    H.w[2] = ~HA;
    H.w[3] = (~LB & 0xFFFFFFFFull) | ((~HB & 0xFFFFFFFFull) << 32);
    uint32_t c[4] = {0, 0, 0, 0};
    count_group(LA, HA, 0x0000FFFFFFFFFFFFull, c);  // chars 0..47
#pragma unroll
    for (int k = 0; k < 4; k++) H.mid[k] = c[k];
    count_group(LA, HA, 0xFFFF000000000000ull, c);  // chars 48..63
    count_group(LB, HB, 0x00000000FFFFFFFFull, c);  // chars 64..95
#pragma unroll
    for (int k = 0; k < 4; k++) H.cnt[k] = c[k];
    return H;
}

__global__ void count4s_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                               uint64_t* __restrict__ super_cnt /* [4][nsuper] */) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t sum[4] = {0, 0, 0, 0};
        for (int r = 0; r < (int)(kSuper4 / 32); r++) {
            const uint64_t j = i * kSuper4 + r * 32 + lane;
            if (j < nblocks) {
                const Half4 a = make_half4(text, n, j * kB4s), b = make_half4(text, n, j * kB4s + kHalf4s);
#pragma unroll
                for (int c = 0; c < 4; c++) sum[c] += a.cnt[c] + b.cnt[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
            if (lane == 0) super_cnt[c * nsuper + i] = sum[c];
        }
    }
}

__global__ void layout4s_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                                const uint64_t* __restrict__ super_base, uint4* __restrict__ lines,
                                uint4* __restrict__ supers) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t running[4];
        uint32_t s[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint64_t base = super_base[c * nsuper + i];
            s[c] = (uint32_t)(base >> kShift4);
            running[c] = base - ((uint64_t)s[c] << kShift4);
        }
        if (lane == 0) supers[i] = make_uint4(s[0], s[1], s[2], s[3]);
        for (int r = 0; r < (int)(kSuper4 / 32); r++) {
            const uint64_t j = i * kSuper4 + r * 32 + lane;
            const bool live = j < nblocks;
            Half4 h0, h1;
            if (live) {
                h0 = make_half4(text, n, j * kB4s);
                h1 = make_half4(text, n, j * kB4s + kHalf4s);
            }
            uint64_t d0 = 0, d1 = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const uint32_t v = live ? h0.cnt[c] + h1.cnt[c] : 0;
                uint32_t incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                if (live) {
                    const uint64_t before = running[c] + (incl - v);          // rank(jB, c) - 2^13 s_{i,c}
                    d0 |= (before + h0.mid[c]) << (16 * c);                   // rank(jB + 48, c) - ...
                    d1 |= (before + h0.cnt[c] + h1.mid[c]) << (16 * c);       // rank(jB + 144, c) - ...
                }
                running[c] += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (live) {
                h0.w[0] = d0;
                h1.w[0] = d1;
                uint4* dst = lines + 4 * j;
                dst[0] = make_uint4((uint32_t)h0.w[0], (uint32_t)(h0.w[0] >> 32), (uint32_t)h0.w[1],
                                    (uint32_t)(h0.w[1] >> 32));
                dst[1] = make_uint4((uint32_t)h0.w[2], (uint32_t)(h0.w[2] >> 32), (uint32_t)h0.w[3],
                                    (uint32_t)(h0.w[3] >> 32));
                dst[2] = make_uint4((uint32_t)h1.w[0], (uint32_t)(h1.w[0] >> 32), (uint32_t)h1.w[1],
                                    (uint32_t)(h1.w[1] >> 32));
                dst[3] = make_uint4((uint32_t)h1.w[2], (uint32_t)(h1.w[2] >> 32), (uint32_t)h1.w[3],
                                    (uint32_t)(h1.w[3] >> 32));
            }
        }
    }
}

// ---------------------------------------------------------------- 128-byte line layout
// sigma 2: line j holds its delta in bits 0..15 and data bits [1008 j, +1008)
// in bits 16..1023.  A warp builds one superblock of 32 lines, one per lane.
struct Line2L {
    uint64_t w[16];
    uint32_t cnt, half;  // ones of the 1008 bits / of their first 504
};

__device__ __forceinline__ Line2L make_line2l(const uint64_t* __restrict__ t, uint64_t n, uint64_t j) {
    Line2L L;
    const uint64_t base = j * kB2L;
    L.w[0] = bits64(t, n, base) << 16;
#pragma unroll
    for (int k = 1; k < 16; k++) L.w[k] = bits64(t, n, base + 64 * k - 16);
    uint32_t h = 0, c = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const uint32_t pc = popc64(L.w[k]);
        c += pc;
        if (k < 8) h += pc;
    }
    L.half = h + popc64(L.w[8] & 0xFFull);  // line bits 16 .. 519 = data bits 0 .. 503
    L.cnt = c;
    return L;
}

__global__ void count2l_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                               uint64_t* __restrict__ super_cnt) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        const uint64_t j = i * kSuper2L + lane;
        uint64_t sum = j < nblocks ? make_line2l(text, n, j).cnt : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) super_cnt[i] = sum;
    }
}

__global__ void layout2l_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                                const uint64_t* __restrict__ super_base, uint4* __restrict__ lines,
                                uint32_t* __restrict__ supers) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        const uint64_t base = super_base[i];
        const uint64_t s = base >> kShift2;
        if (lane == 0) supers[i] = (uint32_t)s;
        const uint64_t j = i * kSuper2L + lane;
        const bool live = j < nblocks;
        Line2L L;
        if (live) L = make_line2l(text, n, j);
        const uint32_t v = live ? L.cnt : 0;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (live) {
            L.w[0] |= (base - (s << kShift2)) + (incl - v) + L.half;  // rank(jB + 504) - 2^11 s_i
            uint4* dst = lines + 8 * j;
#pragma unroll
            for (int k = 0; k < 8; k++)
                dst[k] = make_uint4((uint32_t)L.w[2 * k], (uint32_t)(L.w[2 * k] >> 32), (uint32_t)L.w[2 * k + 1],
                                    (uint32_t)(L.w[2 * k + 1] >> 32));
        }
    }
}

// sigma 4: line j holds chars [480 j, +480): groups g = 0..6 of 64 chars in
// words 2+2g / 3+2g, the 32-char tail in word 1, the deltas in word 0.  A
// warp builds one superblock of 64 lines, two per lane.
struct Line4L {
    uint64_t w[16];
    uint32_t cnt[4], half[4];  // per-symbol counts of the 480 chars / of the first 240
};

__device__ __forceinline__ Line4L make_line4l(const uint64_t* __restrict__ t, uint64_t n, uint64_t j) {
    Line4L R;
    const uint64_t nbits = 2 * n, c0 = j * kB4L;
    uint32_t cnt[4] = {0, 0, 0, 0}, half[4] = {0, 0, 0, 0};
#pragma unroll
    for (int g = 0; g < 7; g++) {
        const uint64_t first = c0 + 64 * g;
        const uint64_t x0 = bits64(t, nbits, 2 * first), x1 = bits64(t, nbits, 2 * first + 64);
        const uint64_t L = (uint64_t)even_bits(x0) | ((uint64_t)even_bits(x1) << 32);
        const uint64_t H = (uint64_t)even_bits(x0 >> 1) | ((uint64_t)even_bits(x1 >> 1) << 32);
        R.w[2 + 2 * g] = ~L;
        R.w[3 + 2 * g] = ~H;
        count_group(L, H, ~0ull, cnt);
        if (g < 3) count_group(L, H, ~0ull, half);
        if (g == 3) count_group(L, H, 0x0000FFFFFFFFFFFFull, half);  // chars 192 .. 239
    }
    const uint64_t x = bits64(t, nbits, 2 * (c0 + 448));
    const uint64_t LB = even_bits(x), HB = even_bits(x >> 1);
    R.w[1] = (~LB & 0xFFFFFFFFull) | ((~HB & 0xFFFFFFFFull) << 32);
    count_group(LB, HB, 0xFFFFFFFFull, cnt);
    R.w[0] = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        R.cnt[c] = cnt[c];
        R.half[c] = half[c];
    }
    return R;
}

__global__ void count4l_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                               uint64_t* __restrict__ super_cnt /* [4][nsuper] */) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t sum[4] = {0, 0, 0, 0};
        for (int r = 0; r < (int)(kSuper4L / 32); r++) {
            const uint64_t j = i * kSuper4L + r * 32 + lane;
            if (j < nblocks) {
                const Line4L L = make_line4l(text, n, j);
#pragma unroll
                for (int c = 0; c < 4; c++) sum[c] += L.cnt[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
            if (lane == 0) super_cnt[c * nsuper + i] = sum[c];
        }
    }
}

__global__ void layout4l_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nsuper,
                                const uint64_t* __restrict__ super_base, uint4* __restrict__ lines,
                                uint4* __restrict__ supers) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nsuper; i += nwarps) {
        uint64_t running[4];
        uint32_t s[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint64_t base = super_base[c * nsuper + i];
            s[c] = (uint32_t)(base >> kShift4);
            running[c] = base - ((uint64_t)s[c] << kShift4);
        }
        if (lane == 0) supers[i] = make_uint4(s[0], s[1], s[2], s[3]);
        for (int r = 0; r < (int)(kSuper4L / 32); r++) {
            const uint64_t j = i * kSuper4L + r * 32 + lane;
            const bool live = j < nblocks;
            Line4L L;
            if (live) L = make_line4l(text, n, j);
            uint64_t d = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const uint32_t v = live ? L.cnt[c] : 0;
                uint32_t incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                if (live) d |= (running[c] + (incl - v) + L.half[c]) << (16 * c);  // rank(jB + 240, c) - 2^13 s
                running[c] += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (live) {
                L.w[0] = d;
                uint4* dst = lines + 8 * j;
#pragma unroll
                for (int k = 0; k < 8; k++)
                    dst[k] = make_uint4((uint32_t)L.w[2 * k], (uint32_t)(L.w[2 * k] >> 32), (uint32_t)L.w[2 * k + 1],
                                        (uint32_t)(L.w[2 * k + 1] >> 32));
            }
        }
    }
}

// ---------------------------------------------------------------- inline layouts
// Built in chunks of 128 lines, independent of the L0 blocks (2^22 lines, 2^16
// for QuadRank24_8): the counts of every chunk, an exclusive scan of them,
// then every chunk's lines, their values relative to the rank at the start of
// their L0 block (that rank is the scanned base of the block's first chunk,
// which also writes it to the L0 table).
constexpr uint64_t kChunkLines = 128;
constexpr uint64_t kChunksPerL0 = kL0Lines / kChunkLines;
constexpr uint64_t kChunksPerL0_24 = kL0Lines24 / kChunkLines;

// sigma 2, VAR 0 = BiRank32 (one value + 480 data bits), VAR 1 = BiRank32x2
// (per 32-byte half: one value + 224 data bits): the line's words with their
// value bits still 0, its count, and the counts before each value's position
// (mid[h]; half0 = the count of half 0 for VAR 1).
struct LineIn2 {
    uint64_t w[8];
    uint32_t cnt, half0, mid[2];
};

template <int VAR>
__device__ __forceinline__ LineIn2 make_line_in2(const uint64_t* __restrict__ t, uint64_t n, uint64_t j) {
    LineIn2 L;
    L.half0 = 0;
    if (VAR == 0) {
        const uint64_t base = j * kB2w;  // data bit d at line bit 32 + d
        L.w[0] = bits64(t, n, base) << 32;
#pragma unroll
        for (int k = 1; k < 8; k++) L.w[k] = bits64(t, n, base + 64 * k - 32);
        // data bits [0, 240) = line bits [32, 272)
        L.mid[0] = popc64(L.w[0]) + popc64(L.w[1]) + popc64(L.w[2]) + popc64(L.w[3]) + popc64(L.w[4] & 0xFFFFull);
        L.mid[1] = 0;
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) c += popc64(L.w[k]);
        L.cnt = c;
    } else {
        uint32_t total = 0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint64_t base = j * kB2x + h * kHalf2x;  // data bit d of the half at half bit 32 + d
            L.w[4 * h] = bits64(t, n, base) << 32;
#pragma unroll
            for (int k = 1; k < 4; k++) L.w[4 * h + k] = bits64(t, n, base + 64 * k - 32);
            // data bits [0, 112) of the half = half bits [32, 144)
            L.mid[h] = popc64(L.w[4 * h]) + popc64(L.w[4 * h + 1]) + popc64(L.w[4 * h + 2] & 0xFFFFull);
            const uint32_t hc = popc64(L.w[4 * h]) + popc64(L.w[4 * h + 1]) + popc64(L.w[4 * h + 2]) +
                                popc64(L.w[4 * h + 3]);
            if (h == 0) L.half0 = hc;
            total += hc;
        }
        L.cnt = total;
    }
    return L;
}

template <int VAR>
__global__ void count_in2_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nchunks,
                                 uint64_t* __restrict__ chunk_cnt) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nchunks; i += nwarps) {
        uint64_t sum = 0;
        for (int r = 0; r < (int)(kChunkLines / 32); r++) {
            const uint64_t j = i * kChunkLines + r * 32 + lane;
            if (j < nblocks) sum += make_line_in2<VAR>(text, n, j).cnt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) chunk_cnt[i] = sum;
    }
}

template <int VAR>
__global__ void layout_in2_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nchunks,
                                  const uint64_t* __restrict__ chunk_base, uint4* __restrict__ lines,
                                  uint64_t* __restrict__ l0tab) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nchunks; i += nwarps) {
        const uint64_t base = chunk_base[i];
        const uint64_t l0 = chunk_base[i & ~(kChunksPerL0 - 1)];  // rank at the start of the L0 block
        if (lane == 0 && (i & (kChunksPerL0 - 1)) == 0) l0tab[i / kChunksPerL0] = base;
        uint64_t running = base - l0;  // < 2^22 * 480
        for (int r = 0; r < (int)(kChunkLines / 32); r++) {
            const uint64_t j = i * kChunkLines + r * 32 + lane;
            LineIn2 L;
            const bool live = j < nblocks;
            if (live) L = make_line_in2<VAR>(text, n, j);
            const uint32_t v = live ? L.cnt : 0;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const uint64_t before = running + (incl - v);  // rank(line start) - rank(L0 start)
            if (live) {
                L.w[0] |= before + L.mid[0];                      // < 2^32
                if (VAR == 1) L.w[4] |= before + L.half0 + L.mid[1];
                uint4* dst = lines + 4 * j;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    dst[k] = make_uint4((uint32_t)L.w[2 * k], (uint32_t)(L.w[2 * k] >> 32), (uint32_t)L.w[2 * k + 1],
                                        (uint32_t)(L.w[2 * k + 1] >> 32));
            }
            running += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// sigma 4: 192 chars as three transposed groups of 64 (words 2 + 2g, 3 + 2g),
// the per-symbol counts of the line and of its first 96 chars (QuadRank32,
// Q24 false) or its first 64 chars (QuadRank24_8, Q24 true).
struct LineIn4 {
    uint64_t w[8];
    uint32_t cnt[4], mid[4];
};

template <bool Q24>
__device__ __forceinline__ LineIn4 make_line_in4(const uint64_t* __restrict__ t, uint64_t n, uint64_t j) {
    LineIn4 R;
    const uint64_t nbits = 2 * n;
    const uint64_t c0 = j * kB4w;
    uint32_t cnt[4] = {0, 0, 0, 0}, mid[4] = {0, 0, 0, 0};
    R.w[0] = R.w[1] = 0;
#pragma unroll
    for (int g = 0; g < 3; g++) {
        const uint64_t first = c0 + 64 * g;
        const uint64_t x0 = bits64(t, nbits, 2 * first), x1 = bits64(t, nbits, 2 * first + 64);
        const uint64_t L = (uint64_t)even_bits(x0) | ((uint64_t)even_bits(x1) << 32);
        const uint64_t H = (uint64_t)even_bits(x0 >> 1) | ((uint64_t)even_bits(x1 >> 1) << 32);
        count_group(L, H, ~0ull, cnt);
        if (g == 0) count_group(L, H, ~0ull, mid);
        if (g == 1 && !Q24) count_group(L, H, 0xFFFFFFFFull, mid);  // chars 64 .. 95
        R.w[2 + 2 * g] = ~L;
        R.w[3 + 2 * g] = ~H;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        R.cnt[c] = cnt[c];
        R.mid[c] = mid[c];
    }
    return R;
}

template <bool Q24>
__global__ void count_in4_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nchunks,
                                 uint64_t* __restrict__ chunk_cnt /* [4][nchunks] */) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nchunks; i += nwarps) {
        uint64_t sum[4] = {0, 0, 0, 0};
        for (int r = 0; r < (int)(kChunkLines / 32); r++) {
            const uint64_t j = i * kChunkLines + r * 32 + lane;
            if (j < nblocks) {
                const LineIn4 L = make_line_in4<Q24>(text, n, j);
#pragma unroll
                for (int c = 0; c < 4; c++) sum[c] += L.cnt[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
            if (lane == 0) chunk_cnt[c * nchunks + i] = sum[c];
        }
    }
}

// QuadRank32: value v_c = rank(192 j + 96, c) - L0_c in word c / 2, half c % 2.
// QuadRank24_8: a_c = rank(192 j + 64, c) - L0_c (< 2^16 * 192 < 2^24) and
// b_c = the count of c in chars 64 .. 191 (<= 128), as a_c | b_c << 24 in the
// same place.
template <bool Q24>
__global__ void layout_in4_kernel(const uint64_t* __restrict__ text, uint64_t n, uint64_t nblocks, uint64_t nchunks,
                                  const uint64_t* __restrict__ chunk_base /* [4][nchunks] */,
                                  uint4* __restrict__ lines, uint64_t* __restrict__ l0tab /* [nl0][4] */) {
    constexpr uint64_t kPer = Q24 ? kChunksPerL0_24 : kChunksPerL0;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < nchunks; i += nwarps) {
        uint64_t running[4];
        const uint64_t first = i & ~(kPer - 1);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint64_t base = chunk_base[c * nchunks + i];
            running[c] = base - chunk_base[c * nchunks + first];
            if (lane == 0 && i == first) l0tab[4 * (i / kPer) + c] = base;
        }
        for (int r = 0; r < (int)(kChunkLines / 32); r++) {
            const uint64_t j = i * kChunkLines + r * 32 + lane;
            const bool live = j < nblocks;
            LineIn4 L;
            if (live) L = make_line_in4<Q24>(text, n, j);
            uint64_t val[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const uint32_t v = live ? L.cnt[c] : 0;
                uint32_t incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                val[c] = running[c] + (incl - v) + (live ? L.mid[c] : 0);  // rank(192 j + 96 or 64, c) - L0
                if (Q24 && live) val[c] |= (uint64_t)(L.cnt[c] - L.mid[c]) << 24;
                running[c] += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (live) {
                L.w[0] = val[0] | (val[1] << 32);
                L.w[1] = val[2] | (val[3] << 32);
                uint4* dst = lines + 4 * j;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    dst[k] = make_uint4((uint32_t)L.w[2 * k], (uint32_t)(L.w[2 * k] >> 32), (uint32_t)L.w[2 * k + 1],
                                        (uint32_t)(L.w[2 * k + 1] >> 32));
            }
        }
    }
}

unsigned grid_for_warps(uint64_t nwarps) {
    uint64_t blocks = (nwarps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const uint64_t cap = (uint64_t)device_props().sms * 64;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    return (unsigned)blocks;
}

}  // namespace

// The inline layouts: chunk counts, scans, lines and the L0 table.
int build_inline_index(qr_index* idx, const uint64_t* d_text, cudaStream_t s) {
    const uint64_t nchunks = (idx->nblocks + kChunkLines - 1) / kChunkLines;
    const int nsym = idx->sigma == 2 ? 1 : 4;
    uint64_t* cnt = nullptr;
    uint64_t* base = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&cnt, sizeof(uint64_t) * nchunks * nsym, s));
    cudaError_t e = cudaMallocAsync((void**)&base, sizeof(uint64_t) * nchunks * nsym, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(cnt, s);
        return cuda_fail(e, "cudaMallocAsync(scan)");
    }
    const unsigned grid = grid_for_warps(nchunks);
    const unsigned threads = 32 * kWarpsPerBlock;
    int rc = QR_OK;
    uint64_t* l0 = (uint64_t*)idx->supers;
    if (idx->sigma == 2) {
        const bool x2 = idx->layout == QR_LAYOUT_INLINE32X2;
        if (x2) count_in2_kernel<1><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, cnt);
        else count_in2_kernel<0><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, cnt);
        rc = exclusive_scan_u64(cnt, base, nchunks, s);
        if (rc == QR_OK && x2)
            layout_in2_kernel<1><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, base, idx->lines, l0);
        else if (rc == QR_OK)
            layout_in2_kernel<0><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, base, idx->lines, l0);
    } else {
        const bool q24 = idx->layout == QR_LAYOUT_INLINE24_8;
        if (q24) count_in4_kernel<true><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, cnt);
        else count_in4_kernel<false><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, cnt);
        for (int c = 0; c < 4 && rc == QR_OK; c++)
            rc = exclusive_scan_u64(cnt + c * nchunks, base + c * nchunks, nchunks, s);
        if (rc == QR_OK && q24)
            layout_in4_kernel<true><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, base, idx->lines,
                                                            l0);
        else if (rc == QR_OK)
            layout_in4_kernel<false><<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nchunks, base, idx->lines,
                                                             l0);
    }
    cudaError_t le = cudaGetLastError();
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(base, s);
    if (rc != QR_OK) return rc;
    if (le != cudaSuccess) return cuda_fail(le, "inline layout kernels");
    return QR_OK;
}

int build_rank_index(qr_index* idx, const uint64_t* d_text, cudaStream_t s) {
    if (inline_layout(idx->layout)) return build_inline_index(idx, d_text, s);
    const uint64_t nsuper = idx->nsuper;
    const int nsym = idx->sigma == 2 ? 1 : 4;
    uint64_t* cnt = nullptr;
    uint64_t* base = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&cnt, sizeof(uint64_t) * nsuper * nsym, s));
    cudaError_t e = cudaMallocAsync((void**)&base, sizeof(uint64_t) * nsuper * nsym, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(cnt, s);
        return cuda_fail(e, "cudaMallocAsync(scan)");
    }
    const unsigned grid = grid_for_warps(nsuper);
    const unsigned threads = 32 * kWarpsPerBlock;
    int rc = QR_OK;
    const bool sector = idx->layout == QR_LAYOUT_SECTOR;
    const bool line128 = idx->layout == QR_LAYOUT_LINE128;
    if (line128) {
        if (idx->sigma == 2) {
            count2l_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, cnt);
            rc = exclusive_scan_u64(cnt, base, nsuper, s);
            if (rc == QR_OK)
                layout2l_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, base, idx->lines,
                                                         (uint32_t*)idx->supers);
        } else {
            count4l_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, cnt);
            for (int c = 0; c < 4 && rc == QR_OK; c++)
                rc = exclusive_scan_u64(cnt + c * nsuper, base + c * nsuper, nsuper, s);
            if (rc == QR_OK)
                layout4l_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, base, idx->lines,
                                                         (uint4*)idx->supers);
        }
    } else if (idx->sigma == 2) {
        if (sector) count2s_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, cnt);
        else count2_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, cnt);
        rc = exclusive_scan_u64(cnt, base, nsuper, s);
        if (rc == QR_OK && sector)
            layout2s_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, base, idx->lines,
                                                     (uint32_t*)idx->supers);
        else if (rc == QR_OK)
            layout2_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, base, idx->lines,
                                                    (uint32_t*)idx->supers);
    } else {
        if (sector) count4s_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, cnt);
        else count4_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, cnt);
        for (int c = 0; c < 4 && rc == QR_OK; c++)
            rc = exclusive_scan_u64(cnt + c * nsuper, base + c * nsuper, nsuper, s);
        if (rc == QR_OK && sector)
            layout4s_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, base, idx->lines,
                                                     (uint4*)idx->supers);
        else if (rc == QR_OK)
            layout4_kernel<<<grid, threads, 0, s>>>(d_text, idx->n, idx->nblocks, nsuper, base, idx->lines,
                                                    (uint4*)idx->supers);
    }
    cudaError_t le = cudaGetLastError();
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(base, s);
    if (rc != QR_OK) return rc;
    if (le != cudaSuccess) return cuda_fail(le, "rank layout kernels");
    return QR_OK;
}

}  // namespace qr
