// Declarations shared by the batched rank kernels of the layouts
// (qr_rank.cu: paper and sector layouts, chains, probe; qr_rank_line.cu:
// 128-byte line layout; qr_rank_in32.cu: the 32-bit inline layouts).
#pragma once

#include "qr_common.cuh"

namespace qr {

enum Kind { kBiScalar = 0, kBiVec = 1, kQuadScalar = 2, kQuadVec = 3, kQuad4 = 4, kQuadPrefix = 5 };

// rank_4 and prefix_rank both need all four counts of the query's line
template <int KIND>
__host__ __device__ constexpr bool all4() { return KIND == kQuad4 || KIND == kQuadPrefix; }

struct RankArgs {
    const uint4* __restrict__ lines;
    const void* __restrict__ supers;
    uint64_t n;
    const uint64_t* __restrict__ q;
    const uint8_t* __restrict__ cvec;
    int c;
    uint64_t m;
    uint64_t* __restrict__ out;
    uint32_t* status;
    // set when region batching was chosen by the automatic rule: the kernel
    // runs only when *gate <= gate_limit (a clustered batch)
    const unsigned long long* gate;
    unsigned long long gate_limit;
};

using KernelFn = void (*)(RankArgs);

// Kernel of the 128-byte line layout for a query kind and K queries per
// thread (K = 1 or 2; nullptr otherwise).
KernelFn pick_line_kind(int kind, int k);

// Dependent queries: the next position of a chain from the last position and
// its rank, uniform in [0, n]: floor(x (n + 1) / 2^64) with
// x = (q + r) * 0x9E3779B97F4A7C15 mod 2^64.
__device__ __forceinline__ uint64_t chain_next(uint64_t q, uint64_t r, uint64_t n) {
    return mulhi64((q + r) * 0x9E3779B97F4A7C15ull, n + 1);
}

// Chain kernel of the 128-byte line layout; a.q = starts, a.m = chains,
// a.out = 2 values per chain (see qr_rank_chain).  Launched with whole warps.
using ChainFn = void (*)(RankArgs, uint64_t);
ChainFn pick_chain_line(bool quad);

// Kernels of the inline layouts (qr_rank_in32.cu) for layout
// QR_LAYOUT_INLINE32, _INLINE32X2 or _INLINE24_8; nullptr where the layout
// has no such kernel (BiRank32x2 is sigma 2 only, QuadRank24_8 sigma 4 only).
KernelFn pick_in32_kind(int kind, int k, int layout);
ChainFn pick_chain_in32(bool quad, int layout);

}  // namespace qr
