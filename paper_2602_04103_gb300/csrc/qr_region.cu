// Region-batched rank: a large batch of queries is grouped by text region
// before it is answered, so that every region of the index is read from HBM
// about once per batch and its lines are then served from L2.
//
// On GB300 a random 64-byte line costs a whole 128-byte DRAM fill, and random
// fills arrive at ~38 G/s, far below the rate at which the same DRAM streams.
// A batch of m uniform queries over an index of L lines touches each line
// about m / L times (2^28 queries over the 3.5e7 lines of a 2^34-bit
// BiRank16 index: 7.75 times), so for such batches it pays to move the
// queries instead of the lines.  Every query is still answered from its own
// line by the paper's query arithmetic (Sec. 3 Eq. 1, Sec. 4 rank1 and
// rank_4); only the order in which lines are visited changes, so results are
// identical.
//
// Passes over a batch cut into tiles of 8192 queries and at most 256 regions
// (region = q >> shift, at least the smallest shift that maps [0, n] onto 256,
// and one more where longer regions pay, see region_extra; n = 2^34 bits
// gives 129 regions of 2^27 positions; the path needs shift <= 29, i.e.
// n < 2^37):
//   sort    tile t sorts its queries by region in shared memory (a counting
//           sort) and writes them back to its own slice of two arrays: a
//           4-byte key (the position inside its region, its symbol, a bad
//           flag) and a 2-byte index inside the tile (with the symbol and
//           the flag again); the start and length of each region's run go to
//           a region-major segment table, seg[r * tiles + t];
//   base    rank and prefix_rank only: the result at the first position of
//           every region, for every symbol (1024 queries);
//   rank    warps take steps of 16 segments of the table, in table order,
//           from a device work queue, i.e. region after region, so the lines
//           of the two or three regions in flight stay in L2 (only the
//           regions that can hold a valid query: out-of-range queries sit in
//           the last region and are never answered); rank and
//           prefix_rank replace each key by the low 32 bits of its result,
//           rank_4 writes the low 32 bits of its four counts (16 bytes) at
//           the key's place in an array of its own;
//   unsort  tile t reads its slice back, restores every result from its low
//           32 bits and its region's base (results of one region differ from
//           the base by less than 2^29), puts it at its index in shared
//           memory and writes the tile's outputs in order.
// Per query that moves 8 (q) + 6 bytes in the sort, 4 + 4 in the rank pass
// and 6 + 8 in the unsort (rank_4: 4 + 16 and 18 + 32), plus the index once
// per batch.  Writing rank_4's rows straight from the rank pass was measured
// and dropped: a scattered 32-byte row, even written by one 32-byte store,
// made the L2 read ~99 bytes from DRAM per query (ncu, 2^24 queries over
// 2^30 characters) against the ~27 the pass needs.  The sort and unsort
// passes read and write whole tiles (coalesced); the rank pass reads runs of
// ~64 keys per (region, tile).  The
// scratch arrays come from a memory pool of the library that keeps them for
// later calls.  Measured on GB300 and kept out: a count pass plus a global
// scan to place runs region-major (one more read of the queries, and
// __match_any_sync grouping ran at 1.2 TB/s); blocks walking 64 runs with a
// shared-memory search (barrier-bound); strided warp steps (warps drift
// apart, the regions in flight outgrow L2); bulk L2 prefetch
// (cp.async.bulk.prefetch.L2) of the next region's lines and of the next
// runs (slower).
//
// Sorted batches: each tile is one run, so a warp step would hold whole
// tiles; such batches are sent to the direct kernels by the probe (see Gate).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "qr_common.cuh"
#include "qr_rank.cuh"

namespace qr {
namespace {

constexpr uint32_t kTile = 8192;    // queries per tile
constexpr uint32_t kRegions = 256;  // regions of the text
constexpr int kPassThreads = 512;   // sort / unsort
constexpr int kPassBlocks = 2;      // resident sort / unsort blocks per SM
constexpr int kPer = kTile / kPassThreads;
constexpr int kRankThreads = 256;

// Key (4 bytes, written by the sort, read by the rank pass): bits 0..28 the
// position inside its region (q - (region << shift) < 2^shift <= 2^29), bit 29
// set for a query that is out of range (q > n) or has a bad symbol, bits
// 30..31 the symbol.  The rank pass of rank / prefix_rank overwrites it with
// the low 32 bits of the result.
// Index (2 bytes): bits 0..12 the index inside the tile, 13..14 the symbol,
// bit 15 the bad flag.
constexpr int kMaxShift = 29;
constexpr uint32_t kKeyBad = 1u << 29;
constexpr int kKeySymShift = 30;
constexpr uint16_t kIdxBad = 0x8000;
constexpr int kIdxSymShift = 13;
constexpr uint32_t kAll = 0xffffffffu;
constexpr int kBaseSyms = 4;  // base table: kRegions x 4 symbols of uint64

__device__ __forceinline__ uint32_t make_key(uint64_t q, uint32_t c, bool bad, int shift) {
    return bad ? kKeyBad : (uint32_t)(q & ((1ull << shift) - 1)) | (c << kKeySymShift);
}
__device__ __forceinline__ uint16_t make_idx(uint32_t i, uint32_t c, bool bad) {
    return (uint16_t)(i | ((c & 3u) << kIdxSymShift) | (bad ? kIdxBad : 0u));
}

__device__ __forceinline__ uint32_t region_of(uint64_t q, int shift) {
    const uint64_t r = q >> shift;
    return r < kRegions ? (uint32_t)r : kRegions - 1;
}

// Exclusive scan of v over the first 32 * nw threads of a block (nw <= 8
// warps); ws = 8 words of shared scratch; *total (may be NULL) receives the
// sum.  Every thread of the block must call it.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, int nw, uint32_t* ws, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += u;
    }
    if (w < nw && lane == 31) ws[w] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int k = 0; k < nw; k++) {
        const uint32_t x = ws[k];
        before += k < w ? x : 0u;
        all += x;
    }
    if (total) *total = all;
    __syncthreads();
    return before + incl - v;
}

// ---------------------------------------------------------------- gate
// With region batching chosen by the automatic rule, a probe kernel counts
// the distinct regions among the first queries of a few tiles spread over
// the batch.  Few regions per tile mean a clustered (e.g. sorted) batch, which
// the direct kernels answer faster (neighbouring queries share lines); the
// direct kernel and the three region passes are all launched, and each reads
// the count first and returns at once unless it is the path chosen.
// gate == NULL: no probe, run unconditionally.
// abort: set by the sort pass when one of its bounded waits expires (its
// work array is then incomplete), so that the rank and unsort passes return
// at once instead of reading it.
struct Gate {
    const unsigned long long* count;
    unsigned long long limit;  // clustered when *count <= limit
    unsigned long long* abort;
};
__device__ __forceinline__ bool regions_chosen(const Gate& g) {
    return (!g.count || *g.count > g.limit) && !(g.abort && *(volatile unsigned long long*)g.abort);
}

constexpr int kProbeTiles = 64;     // tiles probed
constexpr int kProbeQueries = 1024; // leading queries of each probed tile
constexpr int kClusterMax = 4;      // mean distinct regions per probe at most -> direct

__global__ void __launch_bounds__(256) region_probe(const uint64_t* __restrict__ q, uint64_t m, int shift,
                                                    uint64_t tiles, unsigned long long* __restrict__ count) {
    __shared__ uint32_t bits[kRegions / 32];
    if (threadIdx.x < kRegions / 32) bits[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t = (uint64_t)blockIdx.x * tiles / gridDim.x, base = t * kTile;
    const uint64_t len = m - base < (uint64_t)kProbeQueries ? m - base : (uint64_t)kProbeQueries;
    for (uint32_t i0 = 0; i0 < kProbeQueries; i0 += blockDim.x) {
        const uint32_t i = i0 + threadIdx.x;
        const uint32_t r = i < len ? region_of(q[base + i], shift) : ~0u;
#pragma unroll
        for (int w = 0; w < (int)(kRegions / 32); w++) {
            const uint32_t mine = (r >> 5) == (uint32_t)w ? 1u << (r & 31) : 0u;
            const uint32_t all = __reduce_or_sync(kAll, mine);
            if ((threadIdx.x & 31) == 0 && all) atomicOr(&bits[w], all);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t c = threadIdx.x < kRegions / 32 ? __popc(bits[threadIdx.x]) : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kAll, c, o);
        if (threadIdx.x == 0) atomicAdd(count, (unsigned long long)c);
    }
}

// ---------------------------------------------------------------- sort
// Counting sort of one tile by region.  The rank of a query inside its region
// comes from a shared-memory atomic; a warp whose queries all fall in one
// region (sorted batches) takes one atomic for all its lanes.  The second
// phase reads the tile's queries again (L2 hits) rather than keeping 16 of
// them per thread in registers across the block-wide scan.  This form (plain
// loads and stores) serves query or symbol arrays that are not 16-byte
// aligned; region_sort_tma below serves the rest.
template <bool VEC>
__global__ void __launch_bounds__(kPassThreads, kPassBlocks) region_sort(const uint64_t* __restrict__ q,
                                                               const uint8_t* __restrict__ cv, uint32_t c0,
                                                               uint32_t sigma, uint64_t m, uint64_t n, int shift,
                                                               uint64_t tiles, uint32_t* __restrict__ keys,
                                                               uint16_t* __restrict__ idxs,
                                                               uint32_t* __restrict__ seg,
                                                               uint32_t* __restrict__ segt, uint32_t* status,
                                                               Gate gate) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* key_st = (uint32_t*)smem;                     // kTile keys in region order
    uint16_t* idx_st = (uint16_t*)(smem + kTile * 4);       // their indices
    uint16_t* rank_in = (uint16_t*)(smem + kTile * 6);      // rank of query i inside its region
    uint32_t* h = (uint32_t*)(smem + kTile * 8);            // region sizes, then starts
    uint32_t* ws = h + kRegions;
    if (!regions_chosen(gate)) return;
    const int lane = threadIdx.x & 31;
    uint32_t flags = 0;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t base = t * kTile;
    const uint32_t len = (uint32_t)(m - base < kTile ? m - base : kTile);
    for (uint32_t r = threadIdx.x; r < kRegions; r += blockDim.x) h[r] = 0;
    __syncthreads();
    {
        uint64_t v[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const uint32_t i = threadIdx.x + k * kPassThreads;
            v[k] = i < len ? q[base + i] : 0;  // default policy: read again below, from L2
        }
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const uint32_t i = threadIdx.x + k * kPassThreads;
            const bool live = i < len;
            const uint32_t r = region_of(v[k], shift);
            const unsigned act = __ballot_sync(kAll, live);
            if (!act) continue;
            const int lead = __ffs(act) - 1;
            const uint32_t r0 = __shfl_sync(kAll, r, lead);
            if (__all_sync(kAll, !live || r == r0)) {
                uint32_t b = 0;
                if (lane == lead) b = atomicAdd(&h[r0], (uint32_t)__popc(act));
                b = __shfl_sync(kAll, b, lead);
                if (live) rank_in[i] = (uint16_t)(b + __popc(act & ((1u << lane) - 1u)));
            } else if (live) {
                rank_in[i] = (uint16_t)atomicAdd(&h[r], 1u);
            }
        }
    }
    __syncthreads();
    const uint32_t sz = threadIdx.x < kRegions ? h[threadIdx.x] : 0u;
    const uint32_t st = block_scan(sz, kRegions / 32, ws, nullptr);
    if (threadIdx.x < kRegions) {
        h[threadIdx.x] = st;
        seg[(uint64_t)threadIdx.x * tiles + t] = st | (sz << 16);
        segt[t * kRegions + threadIdx.x] = st | (sz << 16);
    }
    __syncthreads();
    {
        uint64_t x[kPer];
        uint32_t cw[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const uint32_t i = threadIdx.x + k * kPassThreads;
            x[k] = i < len ? ld_stream_u64(q + base + i) : 0;
            cw[k] = VEC ? (i < len ? (uint32_t)ld_stream_u8(cv + base + i) : 0u) : c0;
        }
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const uint32_t i = threadIdx.x + k * kPassThreads;
            if (i < len) {
                const bool range_bad = x[k] > n, sym_bad = cw[k] >= sigma;
                flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                const uint32_t pos = h[region_of(x[k], shift)] + rank_in[i];
                key_st[pos] = make_key(x[k], cw[k], range_bad || sym_bad, shift);
                idx_st[pos] = make_idx(i, cw[k], range_bad || sym_bad);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        const uint32_t p = threadIdx.x + k * kPassThreads;
        if (p < len) {
            keys[base + p] = key_st[p];
            idxs[base + p] = idx_st[p];
        }
    }
    __syncthreads();  // the next tile reuses the shared arrays
    }
    if (flags) atomicOr(status, flags);
}

constexpr size_t kSortSmem = (size_t)kTile * 8 + (kRegions + 8) * 4;

// ---------------------------------------------------------------- sort with TMA bulk copies
// The same counting sort, with the tile moved by the TMA unit: each block
// (one per SM, 1024 threads) loads the next tile's queries into a second
// shared buffer with one bulk copy (cp.async.bulk, completion counted on an
// mbarrier) while it sorts the current one, copies the tile's per-query
// symbols the same way, reads its queries from shared memory in both phases,
// and writes the sorted tile back with one bulk store.  Needs q, the symbols
// and the work array 16-byte aligned (else region_sort runs); a ragged last
// tile is read and written by the threads.  Every wait on an mbarrier is
// bounded: on expiry the kernel sets the timeout status bit, waits (again
// bounded) for its own copies and returns.  Measured (2^28 queries): 0.92 ms
// against 1.11 for region_sort (sigma 2), 0.95 against 1.24 with per-query
// symbols.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// A wait gives up after 0.25 s of the GPU's global timer (a 64 KB copy takes
// microseconds) or 2^26 polls, whichever comes first.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t kWaitNs = 250000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
    for (int k = 0; k < 8; k++)
        if (mbar_wait_bounded(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

constexpr int kTmaThreads = 1024;             // one block per SM: more warps hide the shared-memory latency
constexpr int kTmaPer = kTile / kTmaThreads;
// queries (two buffers) + keys + indices + ranks inside the regions + symbols
// (two buffers) + region sizes, the scan's scratch and two mbarriers
constexpr size_t kSortTmaSmem = (size_t)kTile * 8 * 2 + (size_t)kTile * 4 + (size_t)kTile * 2 + (size_t)kTile * 2 +
                                (size_t)kTile * 2 + (kRegions + 8) * 4 + 16;
static_assert(kSortTmaSmem <= 227 * 1024 - 64, "sort pass: shared memory above the per-block limit");

// Full tiles take a branch-free form of the region count that keeps each
// item's region and its rank inside the region in registers, so that the
// shared-memory atomics, and later the scatter, of a thread's items overlap
// (0.82 against 0.91 ms per 2^28 queries with a branch per item).
template <bool VEC>
__global__ void __launch_bounds__(kTmaThreads, 1) region_sort_tma(const uint64_t* __restrict__ q,
                                                                   const uint8_t* __restrict__ cv, uint32_t c0,
                                                                   uint32_t sigma, uint64_t m, uint64_t n, int shift,
                                                                   uint64_t tiles, uint32_t* __restrict__ keys,
                                                                   uint16_t* __restrict__ idxs,
                                                                   uint32_t* __restrict__ seg,
                                                                   uint32_t* __restrict__ segt, uint32_t* status,
                                                                   Gate gate, int withhold) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* raw0 = (uint64_t*)smem;                        // queries of the tile, in order (two buffers)
    uint64_t* raw1 = raw0 + kTile;
    uint32_t* key_st = (uint32_t*)(raw1 + kTile);            // keys in region order
    uint16_t* idx_st = (uint16_t*)(key_st + kTile);          // their indices
    uint16_t* rank_in = idx_st + kTile;                      // rank of query i inside its region
    uint8_t* csym0 = (uint8_t*)(rank_in + kTile);            // per-query symbols of the tile (VEC, two buffers)
    uint8_t* csym1 = csym0 + kTile;
    uint32_t* h = (uint32_t*)(csym1 + kTile);                // region sizes, then starts
    uint32_t* ws = h + kRegions;
    uint64_t* bar = (uint64_t*)(ws + 8);                     // one mbarrier per buffer pair (queries, symbols)
    __shared__ int s_abort;
    if (!regions_chosen(gate)) return;
    const int lane = threadIdx.x & 31;
    auto full = [&](uint64_t t) { return t < tiles && (t + 1) * kTile <= m; };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    uint64_t t = blockIdx.x;
    // withhold (test hook): block 0 never issues its first load, so its first
    // wait runs out and the timeout path is taken
    constexpr uint32_t kTileBytes = kTile * 8 + (VEC ? kTile : 0);  // one tile's queries (and symbols)
    if (threadIdx.x == 0 && full(t) && !(withhold && blockIdx.x == 0)) {
        mbar_expect_tx(&bar[0], kTileBytes);
        bulk_load(raw0, q + t * kTile, kTile * 8, &bar[0]);
        if (VEC) bulk_load(csym0, cv + t * kTile, kTile, &bar[0]);
    }
    uint32_t flags = 0, j = 0;
    bool pending = false;  // thread 0: a load issued into the other buffer and not yet waited for
    // thread 0: the load of the current tile's buffer was issued (only the
    // test hook's first tile has none)
    bool issued = full(t) && !(withhold && blockIdx.x == 0);
    for (; t < tiles; t += gridDim.x, j++) {
        const uint32_t b = j & 1;
        uint64_t* raw = b ? raw1 : raw0;
        uint8_t* csym = b ? csym1 : csym0;
        const uint64_t base = t * kTile;
        const uint32_t len = (uint32_t)(m - base < kTile ? m - base : kTile);
        const uint64_t tn = t + gridDim.x;
        if (threadIdx.x == 0) {
            if (j > 0) issued = pending;
            pending = false;
            if (full(tn)) {  // the other buffers were last read before the previous iteration's final barrier
                fence_proxy_async();
                mbar_expect_tx(&bar[b ^ 1], kTileBytes);
                bulk_load(b ? raw0 : raw1, q + tn * kTile, kTile * 8, &bar[b ^ 1]);
                if (VEC) bulk_load(b ? csym0 : csym1, cv + tn * kTile, kTile, &bar[b ^ 1]);
                pending = true;
            }
            if (full(t) && !mbar_wait_bounded(&bar[b], (j >> 1) & 1)) {
                atomicOr(status, kStatusTimeout);
                if (gate.abort) *(volatile unsigned long long*)gate.abort = 1;
                s_abort = 1;
            }
        }
        if (!full(t)) {
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) raw[i] = q[base + i];
            if (VEC)
                for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) csym[i] = cv[base + i];
        }
        for (uint32_t r = threadIdx.x; r < kRegions; r += blockDim.x) h[r] = 0;
        __syncthreads();
        if (s_abort) break;
        if (full(t) && threadIdx.x != 0) mbar_try_wait(&bar[b], (j >> 1) & 1);  // (completed: acquire the data)
        const bool pipe = len == kTile;
        // (pipe) region of each item | its rank inside the region << 8; with one
        // symbol for the batch also its position inside the region |
        // out-of-range bit, so that the scatter reads no query again (with
        // per-query symbols the extra registers cost more than the read)
        uint32_t rr[kTmaPer], wq[kTmaPer];
        if (pipe) {
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) {
                const uint64_t x = raw[threadIdx.x + k * kTmaThreads];
                rr[k] = region_of(x, shift);
                if (!VEC) wq[k] = x > n ? kKeyBad : (uint32_t)(x & ((1ull << shift) - 1));
            }
            // a warp whose items all share one region (a clustered tile) takes
            // 32 places per atomic; otherwise every item takes its own.  One
            // vote for all the items keeps the shuffle and vote traffic off the
            // shared-memory pipe this pass is bound by.
            const uint32_t r0 = __shfl_sync(kAll, rr[0], 0);
            bool same = true;
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) same &= rr[k] == r0;
            if (__all_sync(kAll, same)) {
#pragma unroll
                for (int k = 0; k < kTmaPer; k++) {
                    uint32_t v = 0;
                    if (lane == 0) v = atomicAdd(&h[r0], 32u);
                    rr[k] |= (__shfl_sync(kAll, v, 0) + (uint32_t)lane) << 8;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kTmaPer; k++) rr[k] |= atomicAdd(&h[rr[k]], 1u) << 8;
            }
        }
        if (!pipe) {
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) {
                const uint32_t i = threadIdx.x + k * kTmaThreads;
                const bool live = i < len;
                const uint32_t r = region_of(live ? raw[i] : 0, shift);
                const unsigned act = __ballot_sync(kAll, live);
                if (!act) continue;
                const int lead = __ffs(act) - 1;
                const uint32_t r0 = __shfl_sync(kAll, r, lead);
                if (__all_sync(kAll, !live || r == r0)) {
                    uint32_t bb = 0;
                    if (lane == lead) bb = atomicAdd(&h[r0], (uint32_t)__popc(act));
                    bb = __shfl_sync(kAll, bb, lead);
                    if (live) rank_in[i] = (uint16_t)(bb + __popc(act & ((1u << lane) - 1u)));
                } else if (live) {
                    rank_in[i] = (uint16_t)atomicAdd(&h[r], 1u);
                }
            }
        }
        __syncthreads();
        const uint32_t sz = threadIdx.x < kRegions ? h[threadIdx.x] : 0u;
        const uint32_t st = block_scan(sz, kRegions / 32, ws, nullptr);
        if (threadIdx.x < kRegions) {
            h[threadIdx.x] = st;
            seg[(uint64_t)threadIdx.x * tiles + t] = st | (sz << 16);
            segt[t * kRegions + threadIdx.x] = st | (sz << 16);
        }
        if (threadIdx.x == 0) bulk_wait_read_all();  // the previous tile's stores have read the staging arrays
        __syncthreads();
        if (pipe) {
            uint32_t pos[kTmaPer], cc[kTmaPer];
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) pos[k] = h[rr[k] & 0xFFu] + (rr[k] >> 8);
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) cc[k] = VEC ? (uint32_t)csym[threadIdx.x + k * kTmaThreads] : c0;
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) {
                const uint32_t i = threadIdx.x + k * kTmaThreads;
                bool range_bad;
                uint32_t w;
                if (VEC) {
                    const uint64_t x = raw[i];
                    range_bad = x > n;
                    w = (uint32_t)(x & ((1ull << shift) - 1));
                } else {
                    range_bad = wq[k] & kKeyBad;
                    w = wq[k];
                }
                const bool sym_bad = cc[k] >= sigma;
                flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                key_st[pos[k]] = range_bad || sym_bad ? kKeyBad : w | (cc[k] << kKeySymShift);
                idx_st[pos[k]] = make_idx(i, cc[k], range_bad || sym_bad);
            }
        }
        if (!pipe) {
#pragma unroll
            for (int k = 0; k < kTmaPer; k++) {
                const uint32_t i = threadIdx.x + k * kTmaThreads;
                if (i < len) {
                    const uint64_t x = raw[i];
                    const uint32_t c = VEC ? (uint32_t)csym[i] : c0;
                    const bool range_bad = x > n, sym_bad = c >= sigma;
                    flags |= (range_bad ? kStatusRange : 0u) | (sym_bad ? kStatusBadSym : 0u);
                    const uint32_t pos = h[region_of(x, shift)] + rank_in[i];
                    key_st[pos] = make_key(x, c, range_bad || sym_bad, shift);
                    idx_st[pos] = make_idx(i, c, range_bad || sym_bad);
                }
            }
        }
        fence_proxy_async();  // this thread's writes to the staging arrays are visible to the bulk stores
        __syncthreads();
        if (len == kTile) {
            if (threadIdx.x == 0) {
                bulk_store(keys + base, key_st, kTile * 4);
                bulk_store(idxs + base, idx_st, kTile * 2);
            }
        } else {
            for (uint32_t p = threadIdx.x; p < len; p += blockDim.x) {
                keys[base + p] = key_st[p];
                idxs[base + p] = idx_st[p];
            }
            __syncthreads();  // the staging arrays are rewritten by the next tile (none: this is the last one)
        }
    }
    if (threadIdx.x == 0) {
        // copies still in flight after a timed-out wait (this tile's load if
        // it was issued, and the next tile's if issued) write this block's
        // shared memory: wait for them before the block exits, up to 8 more
        // bounded waits (2 s) each.  A copy of valid global memory completes
        // well within that; if one did not, the status already holds
        // QR_ETIMEOUT and the context is to be treated as suspect.
        if (s_abort) {
            if (issued) mbar_wait_drain(&bar[j & 1], (j >> 1) & 1);
            if (pending) mbar_wait_drain(&bar[(j & 1) ^ 1], ((j + 1) >> 1) & 1);
        }
        bulk_wait_all();  // every store is complete before the block exits
    }
    if (flags) atomicOr(status, flags);
}


// ---------------------------------------------------------------- unsort
// Tile t's results back in query order.  The rank pass left the low 32 bits
// of each result in place of its key; the result itself is
// base + (low32 - low32(base)) mod 2^32, with base = the result at the first
// position of the query's region for the query's symbol (bases[r * 4 + c]),
// because results of one region exceed their base by less than 2^shift <=
// 2^29.  The region of each sorted place comes from the tile's segment
// entries: every warp writes the region number over the places of its
// regions' runs (reg8; only the first nreg regions, the ones that can hold a
// valid query: the places of out-of-range queries keep a stale region, which
// their UINT64_MAX result ignores), then every thread restores its results
// and puts them at their index inside the tile, and the tile is written out
// in order.
constexpr int kUnsortThreads = 512;
constexpr int kUnsortPer = kTile / kUnsortThreads;
constexpr int kUnsortChunks = kUnsortPer / 4;  // chunks of four consecutive sorted places per thread
constexpr size_t kUnsortSmem = (size_t)kTile * 8 + (size_t)kRegions * kBaseSyms * 8 + (size_t)kRegions * 4 +
                                (size_t)kTile;

__global__ void __launch_bounds__(kUnsortThreads, 2) region_unsort(const uint32_t* __restrict__ keys,
                                                                   const uint16_t* __restrict__ idxs,
                                                                   const uint32_t* __restrict__ segt,
                                                                   const uint64_t* __restrict__ bases, uint64_t m,
                                                                   uint64_t tiles, uint32_t nreg,
                                                                   uint64_t* __restrict__ out, Gate gate) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* res = (uint64_t*)smem;                        // the tile's results in query order
    uint64_t* btab = res + kTile;                           // bases[kRegions * 4]
    uint32_t* tseg = (uint32_t*)(btab + kRegions * kBaseSyms);  // the tile's segment entries
    uint8_t* reg8 = (uint8_t*)(tseg + kRegions);             // region of every sorted place
    if (!regions_chosen(gate)) return;
    for (uint32_t i = threadIdx.x; i < kRegions * kBaseSyms; i += blockDim.x) btab[i] = bases[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this thread's segment entry of the block's next tile, loaded a tile ahead
    uint32_t e_next = 0;
    if (threadIdx.x < kRegions && blockIdx.x < tiles) e_next = __ldg(segt + blockIdx.x * kRegions + threadIdx.x);
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t base = t * kTile;
        const uint32_t len = (uint32_t)(m - base < kTile ? m - base : kTile);
        // the tile's keys and indices first (their DRAM latency overlaps the
        // region fill below), four consecutive places per load: chunk j of
        // this thread holds places 4 (threadIdx.x + 512 j) .. + 3
        uint4 kv[kUnsortChunks];
        uint2 ix[kUnsortChunks];
#pragma unroll
        for (int j = 0; j < kUnsortChunks; j++) {
            const uint32_t p = 4 * (threadIdx.x + j * kUnsortThreads);
            if (p + 4 <= len) {
                kv[j] = ld_stream_v4u32(keys + base + p);
                ix[j] = ld_stream_v2u32((const uint32_t*)(idxs + base + p));
            } else {
                uint32_t k4[4] = {0, 0, 0, 0}, i4[4] = {0, 0, 0, 0};
                for (uint32_t u = 0; u < 4; u++)
                    if (p + u < len) {
                        k4[u] = ld_stream_u32(keys + base + p + u);
                        i4[u] = ld_stream_u16(idxs + base + p + u);
                    }
                kv[j] = make_uint4(k4[0], k4[1], k4[2], k4[3]);
                ix[j] = make_uint2(i4[0] | (i4[1] << 16), i4[2] | (i4[3] << 16));
            }
        }
        if (threadIdx.x < kRegions) {
            tseg[threadIdx.x] = e_next;
            const uint64_t tn = t + gridDim.x;
            if (tn < tiles) e_next = __ldg(segt + tn * kRegions + threadIdx.x);
        }
        __syncthreads();
        for (uint32_t r = warp; r < nreg; r += kUnsortThreads / 32) {
            const uint32_t e = tseg[r];
            const uint32_t st = e & 0xFFFFu, ln = e >> 16;
            for (uint32_t k = lane; k < ln; k += 32) reg8[st + k] = (uint8_t)r;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kUnsortChunks; j++) {
            const uint32_t p = 4 * (threadIdx.x + j * kUnsortThreads);
            const uint32_t rg = *(const uint32_t*)(reg8 + p);   // the regions of the four places
            const uint32_t k4[4] = {kv[j].x, kv[j].y, kv[j].z, kv[j].w};
            const uint32_t i4[4] = {ix[j].x & 0xFFFFu, ix[j].x >> 16, ix[j].y & 0xFFFFu, ix[j].y >> 16};
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (p + u < len) {
                    const uint32_t r = (rg >> (8 * u)) & 0xFFu;
                    const uint64_t b = btab[r * kBaseSyms + ((i4[u] >> kIdxSymShift) & 3u)];
                    const uint64_t v = b + (uint32_t)(k4[u] - (uint32_t)b);
                    res[i4[u] & (kTile - 1)] = (i4[u] & kIdxBad) ? ~0ull : v;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kUnsortPer; k++) {
            const uint32_t i = threadIdx.x + k * kUnsortThreads;
            if (i < len) st_stream_u64(out + base + i, res[i]);
        }
        // the next tile writes tseg and reg8 before its first barrier and res
        // only after its second: every read of this tile is done by then
    }
}

// rank_4: tile t's rows back in query order.  The rank pass left the low 32
// bits of the four counts of every sorted place (16 bytes, res16); each count
// is restored from its region's base for that symbol as in region_unsort.
// The tile's 16-byte rows and their regions are first put at their query
// index in shared memory (128 KiB + 16 KiB: one block of 1024 threads per
// SM), then every thread writes whole 32-byte output rows in order.
constexpr int kUnsort4Threads = 1024;
constexpr int kUnsort4Per = kTile / kUnsort4Threads;
constexpr uint16_t kRowBad = 0x100;  // (qreg) a bad query: a row of UINT64_MAX
constexpr size_t kUnsort4Smem = (size_t)kTile * 16 + (size_t)kTile * 2 + (size_t)kRegions * kBaseSyms * 8 +
                                (size_t)kRegions * 4 + (size_t)kTile;
static_assert(kUnsort4Smem <= 227 * 1024, "rank_4 unsort: shared memory above the per-block limit");

__global__ void __launch_bounds__(kUnsort4Threads, 1) region_unsort4(const uint32_t* __restrict__ res16,
                                                                     const uint16_t* __restrict__ idxs,
                                                                     const uint32_t* __restrict__ segt,
                                                                     const uint64_t* __restrict__ bases, uint64_t m,
                                                                     uint64_t tiles, uint32_t nreg,
                                                                     uint64_t* __restrict__ out4, int out4_32,
                                                                     Gate gate) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* rel = (uint4*)smem;                               // the tile's low 32 bits of the counts, query order
    uint64_t* btab = (uint64_t*)(rel + kTile);               // bases[4][kRegions]
    uint16_t* qreg = (uint16_t*)(btab + kRegions * kBaseSyms);  // region of every query (kRowBad: bad)
    uint32_t* tseg = (uint32_t*)(qreg + kTile);              // the tile's segment entries
    uint8_t* reg8 = (uint8_t*)(tseg + kRegions);             // region of every sorted place
    if (!regions_chosen(gate)) return;
    // bases by symbol, then region: a row's four lookups below then spread
    // over the banks (region-major rows of 32 bytes put every region of a
    // warp on one of four bank groups for each symbol)
    for (uint32_t i = threadIdx.x; i < kRegions * kBaseSyms; i += blockDim.x)
        btab[(i % kBaseSyms) * kRegions + i / kBaseSyms] = bases[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t e_next = 0;
    if (threadIdx.x < kRegions && blockIdx.x < tiles) e_next = __ldg(segt + blockIdx.x * kRegions + threadIdx.x);
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t base = t * kTile;
        const uint32_t len = (uint32_t)(m - base < kTile ? m - base : kTile);
        uint4 rv[kUnsort4Per];
        uint16_t ix[kUnsort4Per];
#pragma unroll
        for (int k = 0; k < kUnsort4Per; k++) {
            const uint32_t p = threadIdx.x + k * kUnsort4Threads;
            rv[k] = p < len ? ld_stream_v4u32(res16 + 4 * (base + p)) : make_uint4(0, 0, 0, 0);
            ix[k] = p < len ? ld_stream_u16(idxs + base + p) : (uint16_t)0;
        }
        if (threadIdx.x < kRegions) {
            tseg[threadIdx.x] = e_next;
            const uint64_t tn = t + gridDim.x;
            if (tn < tiles) e_next = __ldg(segt + tn * kRegions + threadIdx.x);
        }
        __syncthreads();
        for (uint32_t r = warp; r < nreg; r += kUnsort4Threads / 32) {
            const uint32_t e = tseg[r];
            const uint32_t st = e & 0xFFFFu, ln = e >> 16;
            for (uint32_t k = lane; k < ln; k += 32) reg8[st + k] = (uint8_t)r;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kUnsort4Per; k++) {
            const uint32_t p = threadIdx.x + k * kUnsort4Threads;
            if (p < len) {
                const uint32_t i = ix[k] & (kTile - 1);
                rel[i] = rv[k];
                qreg[i] = (ix[k] & kIdxBad) ? kRowBad : (uint16_t)reg8[p];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kUnsort4Per; k++) {
            const uint32_t i = threadIdx.x + k * kUnsort4Threads;
            if (i < len) {
                const uint16_t r = qreg[i];
                uint64_t v[4];
                if (r & kRowBad) {
                    v[0] = v[1] = v[2] = v[3] = ~0ull;
                } else {
                    const uint4 x = rel[i];
                    const uint32_t lo[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const uint64_t b = btab[c * kRegions + r];
                        v[c] = b + (uint32_t)(lo[c] - (uint32_t)b);
                    }
                }
                uint64_t* o = out4 + 4 * (base + i);
                if (out4_32) {
                    st_stream_v4u64(o, v[0], v[1], v[2], v[3]);
                } else {
                    st_stream_v2u64(o, v[0], v[1]);
                    st_stream_v2u64(o + 2, v[2], v[3]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- rank
// Paper layout (BiRank16 / QuadRank16): the 32-byte half of the line that
// holds the query's bits, plus the first 8 or 16 bytes (the deltas) when that
// is the upper half.  Sector layout: the one self-contained half.
// PREFIX (sigma 4): prefix_rank(q, c), the sum of the four counts up to c,
// from all four superblock offsets.
// LAY: the index layout (QR_LAYOUT_PAPER, _SECTOR, _INLINE32, _INLINE32X2,
// _INLINE24_8).  QuadRank24_8 keeps its values and chars 0 .. 63 in the first
// sector: a query there loads that sector alone, the others both.
template <int LAY, bool QUAD, bool PREFIX = false>
struct RegionLoad {
    u64x4 X, X2;     // the sector(s) the query needs (X2: the second sector of an inline line)
    uint64_t w0, w1;
    uint32_t s;
    uint4 s4;
    uint64_t l0;     // inline layouts: the L0 entry (of the query's symbol)
    uint4 l4a, l4b;  // sigma-4 inline layouts, all four symbols: the four L0 entries
    uint32_t pos;
};

// EL: index lines and superblock entries are loaded with an L2 evict-last
// policy (pol), so that they outlive the streaming work items until the
// region's other queries have used them.
template <bool EL>
__device__ __forceinline__ u64x4 ix_ld32(const uint4* p, uint64_t pol) {
    return EL ? ld_line32_hint(p, pol) : ld_line32(p);
}
template <bool EL>
__device__ __forceinline__ uint4 ix_ld16(const uint4* p, uint64_t pol) {
    return EL ? ld_line16_hint(p, pol) : ld_line16(p);
}
template <bool EL>
__device__ __forceinline__ uint32_t ix_ld_u32(const uint32_t* p, uint64_t pol) {
    return EL ? ld_u32_hint(p, pol) : __ldg(p);
}

// N32 (sector and inline layouts, n < 2^37): the line index from a 32-bit
// high multiply, x = q >> 5 (or q >> 6) < 2^32 and the usual magic numbers for
// 15, 3 and 7: ceil(2^35 / 15), ceil(2^33 / 3), ceil(2^34 / 7), exact for every
// 32-bit x.
template <int LAY, bool QUAD, bool PREFIX = false, bool EL = false, bool N32 = false>
__device__ __forceinline__ void region_issue(RegionLoad<LAY, QUAD, PREFIX>& L, const uint4* __restrict__ lines,
                                             const void* __restrict__ supers, uint64_t q, uint32_t c,
                                             uint64_t pol = 0) {
    if (LAY == QR_LAYOUT_INLINE32X2) {  // sigma 2 only
        uint64_t j;
        uint32_t p;
        if (N32) {
            const uint32_t j32 = __umulhi((uint32_t)(q >> 6), 0x92492493u) >> 2;
            j = j32;
            p = (uint32_t)q - j32 * (uint32_t)kB2x;
        } else {
            j = div448(q);
            p = (uint32_t)(q - j * kB2x);
        }
        const uint32_t h = p >= kHalf2x;
        L.pos = p - h * (uint32_t)kHalf2x;
        L.l0 = __ldg((const uint64_t*)supers + (j >> kL0Shift));
        L.X = ix_ld32<EL>(lines + 4 * j + 2 * h, pol);
        L.w0 = L.w1 = 0;
    } else if (LAY == QR_LAYOUT_INLINE24_8) {  // sigma 4 only
        uint64_t j;
        if (N32) {
            const uint32_t j32 = __umulhi((uint32_t)(q >> 6), 0xAAAAAAABu) >> 1;
            j = j32;
            L.pos = (uint32_t)q - j32 * (uint32_t)kB4w;
        } else {
            j = div192(q);
            L.pos = (uint32_t)(q - j * kB4w);
        }
        const uint64_t* l0 = (const uint64_t*)supers + 4 * (j >> kL0Shift24);
        if (PREFIX) {
            L.l4a = __ldg((const uint4*)l0);
            L.l4b = __ldg((const uint4*)l0 + 1);
        } else {
            L.l0 = __ldg(l0 + c);
        }
        L.X = ix_ld32<EL>(lines + 4 * j, pol);
        L.X2 = L.pos >= 64 ? ix_ld32<EL>(lines + 4 * j + 2, pol) : u64x4{0, 0, 0, 0};
        L.w0 = L.w1 = 0;
    } else if (LAY == QR_LAYOUT_INLINE32) {
        uint64_t j;
        if (N32) {
            const uint32_t j32 = QUAD ? __umulhi((uint32_t)(q >> 6), 0xAAAAAAABu) >> 1
                                      : __umulhi((uint32_t)(q >> 5), 0x88888889u) >> 3;
            j = j32;
            L.pos = (uint32_t)q - j32 * (uint32_t)(QUAD ? kB4w : kB2w);
        } else {
            j = QUAD ? div192(q) : div480(q);
            L.pos = (uint32_t)(q - j * (QUAD ? kB4w : kB2w));
        }
        const uint64_t* l0 = (const uint64_t*)supers;
        if (!QUAD) {
            L.l0 = __ldg(l0 + (j >> kL0Shift));
        } else if (PREFIX) {
            L.l4a = __ldg((const uint4*)(l0 + 4 * (j >> kL0Shift)));
            L.l4b = __ldg((const uint4*)(l0 + 4 * (j >> kL0Shift)) + 1);
        } else {
            L.l0 = __ldg(l0 + 4 * (j >> kL0Shift) + c);
        }
        L.X = ix_ld32<EL>(lines + 4 * j, pol);
        L.X2 = ix_ld32<EL>(lines + 4 * j + 2, pol);
        L.w0 = L.w1 = 0;
    } else if (LAY == QR_LAYOUT_SECTOR) {
        uint64_t j;
        uint32_t h;
        if (!QUAD) {
            uint32_t p;
            if (N32) {
                const uint32_t j32 = __umulhi((uint32_t)(q >> 5), 0x88888889u) >> 3;
                j = j32;
                p = (uint32_t)q - j32 * (uint32_t)kB2s;
            } else {
                j = div480(q);
                p = (uint32_t)(q - j * kB2s);
            }
            h = p >= kHalf2s;
            L.pos = p - h * (uint32_t)kHalf2s;
            L.s = ix_ld_u32<EL>((const uint32_t*)supers + (j >> 7), pol);
        } else {
            uint32_t d;
            if (N32) {
                const uint32_t j32 = __umulhi((uint32_t)(q >> 6), 0xAAAAAAABu) >> 1;
                j = j32;
                d = (uint32_t)q - j32 * (uint32_t)kB4s;
            } else {
                j = div192(q);
                d = (uint32_t)(q - j * kB4s);
            }
            h = d >= kHalf4s;
            L.pos = d - h * (uint32_t)kHalf4s;
            if (PREFIX) L.s4 = __ldg((const uint4*)supers + (j >> 8));
            else L.s = ix_ld_u32<EL>((const uint32_t*)supers + 4 * (j >> 8) + c, pol);
        }
        L.X = ix_ld32<EL>(lines + 4 * j + 2 * h, pol);
        L.w0 = L.w1 = 0;
    } else {
        uint64_t j;
        bool upper;
        if (!QUAD) {
            j = div496(q);
            L.pos = (uint32_t)(q - j * kB2);
            upper = L.pos >= kMid2;
            L.s = ix_ld_u32<EL>((const uint32_t*)supers + (j >> 7), pol);
        } else {
            j = div224(q);
            L.pos = (uint32_t)(q - j * kB4) + 32;
            upper = L.pos >= 128;
            if (PREFIX) L.s4 = __ldg((const uint4*)supers + (j >> 8));
            else L.s = ix_ld_u32<EL>((const uint32_t*)supers + 4 * (j >> 8) + c, pol);
        }
        const uint4* P = lines + 4 * j;
        L.X = ix_ld32<EL>(P + 2 * upper, pol);
        L.w0 = L.w1 = 0;
        if (upper) {
            const uint4 d = ix_ld16<EL>(P, pol);
            L.w0 = lo64(d);
            L.w1 = hi64(d);
        }
    }
}

// rank_4: the four counts of a query from the loads of the prefix form (all
// four superblock offsets).
template <int LAY>
__device__ __forceinline__ void region_finish4(const RegionLoad<LAY, true, true>& L, uint64_t r[4]) {
    if (LAY == QR_LAYOUT_INLINE32 || LAY == QR_LAYOUT_INLINE24_8) {
        const uint64_t b[4] = {lo64(L.l4a), hi64(L.l4a), lo64(L.l4b), hi64(L.l4b)};
        if (LAY == QR_LAYOUT_INLINE24_8) quad24_finish4(b, L.X, L.X2, L.pos, r);
        else quad32_finish4(b, L.X, L.X2, L.pos, r);
        return;
    }
    const uint32_t s4[4] = {L.s4.x, L.s4.y, L.s4.z, L.s4.w};
    if (LAY == QR_LAYOUT_SECTOR) {
        quad_sector_finish4(s4, L.X, L.pos, r);
    } else {
        const uint64_t x[4] = {L.X.a, L.X.b, L.X.c, L.X.d};
        const bool upper = L.pos >= 128;
        quad_finish4(s4, upper ? L.w0 : L.X.a, upper ? L.w1 : L.X.b, x, L.pos, r);
    }
}

template <int LAY, bool QUAD, bool PREFIX = false>
__device__ __forceinline__ uint64_t region_finish(const RegionLoad<LAY, QUAD, PREFIX>& L, uint64_t q, uint32_t c) {
    if constexpr (PREFIX) {
        uint64_t r[4];
        region_finish4<LAY>(L, r);
        uint64_t sum = 0;
#pragma unroll
        for (uint32_t k = 0; k < 4; k++) sum += k <= c ? r[k] : 0;
        return sum;
    }
    if (LAY == QR_LAYOUT_INLINE32X2) {
        const uint64_t r1 = in32x2_finish(L.l0, L.X, L.pos);
        return c == 1 ? r1 : q - r1;
    }
    if (LAY == QR_LAYOUT_INLINE24_8) return quad24_finish1(L.l0, L.X, L.X2, L.pos, (int)c);
    if (LAY == QR_LAYOUT_INLINE32) {
        if (!QUAD) {
            const uint64_t r1 = in32_bi_finish(L.l0, L.X, L.X2, L.pos);
            return c == 1 ? r1 : q - r1;
        }
        return quad32_finish1(L.l0, L.X, L.X2, L.pos, (int)c);
    }
    if (LAY == QR_LAYOUT_SECTOR) {
        if (!QUAD) {
            const uint64_t r1 = birank_sector_finish(L.s, L.X, L.pos);
            return c == 1 ? r1 : q - r1;
        }
        return quad_sector_finish1(L.s, L.X, L.pos, (int)c);
    }
    const uint64_t x[4] = {L.X.a, L.X.b, L.X.c, L.X.d};
    if (!QUAD) {
        const bool upper = L.pos >= kMid2;
        const uint64_t r1 = birank_finish(L.s, upper ? L.w0 : L.X.a, x, L.pos);
        return c == 1 ? r1 : q - r1;
    }
    const bool upper = L.pos >= 128;
    const uint64_t w0 = upper ? L.w0 : L.X.a, w1 = upper ? L.w1 : L.X.b;
    return quad_finish1(L.s, quad_delta(w0, w1, (int)c), x, L.pos, (int)c);
}

// Modes of the rank pass: rank(q, c) (scalar or per-query symbol), rank_4,
// prefix_rank(q, c).
constexpr int kModeRank = 0;
constexpr int kModeRank4 = 1;
constexpr int kModePrefix = 2;

// The rank pass.  Every warp walks its own runs of SEGS consecutive
// segments of the region-major table, taking its steps in table order from a
// device work queue (QUEUE) or by a stride: the lengths are scanned with
// shuffles, the runs' keys are laid end to end and each lane answers keys
// lane, lane + 32, ..., K of them per round; the run holding a key is found
// by a log2(SEGS)-step search over the starts held in the lanes.  The keys
// of round t + P are loaded while round t fetches its lines and counts, and
// the table entries of the next step while this step runs.  No shared
// memory, no block barrier.  With the queue the steps in flight stay close
// together in the table, so the regions they touch stay in L2.
template <int K>
struct ItemSlot {
    uint32_t key[K];
    uint32_t at[K];   // place in the key array (m < 2^32)
    uint32_t reg[K];  // region of the key's run
};

template <int K, int SEGS>
__device__ __forceinline__ void fetch_items(ItemSlot<K>& S, const uint32_t* __restrict__ keys, uint32_t j0,
                                            uint32_t total, uint32_t start, uint32_t sbase, uint32_t sreg,
                                            int lane) {
#pragma unroll
    for (int k = 0; k < K; k++) {
        const uint32_t j = j0 + lane + 32 * k;
        // the last segment s with start[s] <= j
        uint32_t sidx = 0;
#pragma unroll
        for (int b = SEGS / 2; b >= 1; b >>= 1) {
            const uint32_t st = __shfl_sync(kAll, start, sidx + b);
            if (st <= j) sidx += b;
        }
        const uint32_t sb = __shfl_sync(kAll, sbase, sidx);
        const uint32_t s0 = __shfl_sync(kAll, start, sidx);
        S.reg[k] = __shfl_sync(kAll, sreg, sidx);
        S.at[k] = sb + (j - s0);
        S.key[k] = j < total ? ld_stream_u32(keys + S.at[k]) : kKeyBad;
    }
}

struct RankPassArgs {
    uint32_t* keys;
    uint32_t* res16;  // rank_4: 4 x 32 bits per sorted place
    const uint32_t* seg;
    uint64_t nseg, tiles;
    const uint4* lines;
    const void* supers;
    uint32_t c0;
    int shift;
    unsigned long long* queue;  // step counter (QUEUE variants), zero at launch
    Gate gate;
};

template <int LAY, bool QUAD, bool VEC, int K, int MINB, int P, int SEGS, bool QUEUE, int MODE = kModeRank,
          bool EL = false, bool N32 = false>
__global__ void __launch_bounds__(kRankThreads, MINB) region_rank(RankPassArgs a) {
    constexpr bool kS4 = MODE != kModeRank;  // loads of all four superblock offsets
    constexpr bool kR4 = MODE == kModeRank4;
    if (!regions_chosen(a.gate)) return;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (kRankThreads / 32);
    constexpr int kWarpSegs = SEGS;
    const uint64_t nsteps = (a.nseg + kWarpSegs - 1) / kWarpSegs;
    constexpr uint32_t kRound = 32 * K;
    uint32_t* __restrict__ keys = a.keys;
    const uint64_t pol = EL ? l2_policy_evict_last() : 0;
    const uint64_t qmask = (1ull << a.shift) - 1;
    // the warp's next step: a strided sequence, or (QUEUE) taken in table order
    // from a device counter, so that the steps in flight stay close together
    auto next_step = [&](uint64_t cur) -> uint64_t {
        if (!QUEUE) return cur + warps;
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(a.queue, 1ull);
        return __shfl_sync(kAll, v, 0);
    };
    uint64_t g = QUEUE ? next_step(0) : (uint64_t)blockIdx.x * (kRankThreads / 32) + (threadIdx.x >> 5);
    // this lane's segment of the warp's current step: length, first key and
    // region (nseg = 256 tiles < 2^27 and m < 2^32: 32-bit arithmetic)
    auto seg_of = [&](uint64_t step, uint32_t& len, uint32_t& sbase, uint32_t& sreg) {
        len = 0;
        sbase = 0;
        sreg = 0;
        const uint64_t w = step * kWarpSegs + lane;
        if (lane < kWarpSegs && step < nsteps && w < a.nseg) {
            const uint32_t e = __ldg(a.seg + w);
            len = e >> 16;
            sreg = (uint32_t)w / (uint32_t)a.tiles;
            sbase = ((uint32_t)w - sreg * (uint32_t)a.tiles) * kTile + (e & 0xFFFFu);
        }
    };
    uint32_t len, sbase, sreg;
    seg_of(g, len, sbase, sreg);
    while (g < nsteps) {
        const uint64_t gn = next_step(g);
        uint32_t nlen, nbase, nreg;
        seg_of(gn, nlen, nbase, nreg);  // the next step's table entries, loaded early
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < kWarpSegs; o <<= 1) {
            const uint32_t u = __shfl_up_sync(kAll, incl, o);
            if (lane >= o) incl += u;
        }
        const uint32_t start = incl - len;  // first key of this lane's segment
        const uint32_t total = __shfl_sync(kAll, incl, kWarpSegs - 1);
        constexpr int PS = P > 0 ? P : 1;
        ItemSlot<K> S[PS];
#pragma unroll
        for (int p = 0; p < P; p++)
            fetch_items<K, SEGS>(S[p], keys, p * kRound, total, start, sbase, sreg, lane);
        for (uint32_t j0 = 0; j0 < total; j0 += kRound) {
            ItemSlot<K> cur;
            if (P == 0) {
                fetch_items<K, SEGS>(cur, keys, j0, total, start, sbase, sreg, lane);
            } else {
                cur = S[0];
#pragma unroll
                for (int p = 0; p + 1 < P; p++) S[p] = S[p + 1];
                if (j0 + P * kRound < total)
                    fetch_items<K, SEGS>(S[PS - 1], keys, j0 + P * kRound, total, start, sbase, sreg, lane);
            }
            RegionLoad<LAY, QUAD, kS4> L[K];
            uint64_t qk[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                const bool bad = cur.key[k] & kKeyBad;
                // bad keys (and idle lanes) read line 0
                qk[k] = bad ? 0 : ((uint64_t)cur.reg[k] << a.shift) | (cur.key[k] & qmask);
                const uint32_t c = VEC ? cur.key[k] >> kKeySymShift : a.c0;
                region_issue<LAY, QUAD, kS4, EL, N32>(L[k], a.lines, a.supers, qk[k], c, pol);
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (kR4) {
                    if constexpr (kR4) {
                        if (cur.key[k] & kKeyBad) continue;
                        uint64_t r[4];
                        region_finish4<LAY>(L[k], r);
                        st_stream_v4u32(a.res16 + 4 * (uint64_t)cur.at[k], (uint32_t)r[0], (uint32_t)r[1],
                                        (uint32_t)r[2], (uint32_t)r[3]);
                    }
                } else {
                    if (cur.key[k] & kKeyBad) continue;
                    const uint32_t c = VEC ? cur.key[k] >> kKeySymShift : a.c0;
                    const uint64_t r = region_finish<LAY, QUAD, kS4>(L[k], qk[k], c);
                    st_stream_u32(keys + cur.at[k], (uint32_t)r);
                }
            }
        }
        len = nlen;
        sbase = nbase;
        sreg = nreg;
        g = gn;
    }
}

// The base table of rank and prefix_rank: bases[r * 4 + c] = the result at
// the first position of region r (r << shift) for symbol c (prefix_rank: up
// to c), by the same query arithmetic as the rank pass; 0 for regions that
// start beyond n (no query falls there) and for c >= sigma.
template <int LAY, bool QUAD, bool PREFIX, bool N32>
__global__ void __launch_bounds__(256) region_base(const uint4* __restrict__ lines, const void* __restrict__ supers,
                                                  uint64_t n, int shift, uint64_t* __restrict__ bases, Gate gate) {
    if (!regions_chosen(gate)) return;
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= kRegions * kBaseSyms) return;
    const uint32_t r = id / kBaseSyms, c = id % kBaseSyms;
    const uint64_t q = (uint64_t)r << shift;
    uint64_t v = 0;
    if (q <= n && (QUAD || c < 2)) {
        RegionLoad<LAY, QUAD, PREFIX> L;
        region_issue<LAY, QUAD, PREFIX, false, N32>(L, lines, supers, q, c, 0);
        v = region_finish<LAY, QUAD, PREFIX>(L, q, c);
    }
    bases[id] = v;
}

// ---------------------------------------------------------------- scratch pool
// One pool per device whose memory stays with the library after a call
// returns it, so that repeated large batches do not map and unmap their
// scratch every time.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

int region_pool(cudaMemPool_t* out) {
    int dev = 0;
    QR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(QR_EINVAL, "region pool: device index");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps p = {};
        p.allocType = cudaMemAllocationTypePinned;
        p.location.type = cudaMemLocationTypeDevice;
        p.location.id = dev;
        cudaMemPool_t pool = nullptr;
        QR_CUDA_TRY(cudaMemPoolCreate(&pool, &p));
        uint64_t keep = ~0ull;
        cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return cuda_fail(e, "region pool: release threshold");
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return QR_OK;
}

template <typename F>
int set_smem(F fn, size_t bytes) {
    QR_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return QR_OK;
}

using RankFn = void (*)(RankPassArgs);
using BaseFn = void (*)(const uint4*, const void*, uint64_t, int, uint64_t*, Gate);

// Rank-pass variants (items per lane and round, resident blocks per SM,
// rounds of items loaded ahead, segments per warp-step, steps from a device
// queue, evict-last index loads).  Measured on GB300 with 8-byte work items
// (2^28 uniform queries, sector layout): 0 1.78 ms, 1 2.11 ms, 2 1.78 ms,
// 3 1.91 ms.
template <int LAY, bool QUAD, bool VEC, bool N32 = false>
RankFn pick_variant(int v) {
    switch (v) {
        case 0: return region_rank<LAY, QUAD, VEC, 2, 4, 1, 16, true, kModeRank, false, N32>;
        case 1: return region_rank<LAY, QUAD, VEC, 1, 6, 2, 16, true, kModeRank, false, N32>;
        case 2: return region_rank<LAY, QUAD, VEC, 2, 4, 1, 16, true, kModeRank, true, N32>;
        case 3: return region_rank<LAY, QUAD, VEC, 4, 3, 1, 16, true, kModeRank, false, N32>;
        default: return nullptr;
    }
}

// The rank pass of one layout: mode kModeRank4 / kModePrefix are sigma 4,
// one symbol or none, default variant; n32: n < 2^37 on a layout with a
// 32-bit line-index division (sector and inline layouts).
template <int LAY>
RankFn pick_rank_lay(bool quad, bool vec, int v, int mode, bool n32) {
    constexpr bool kN32 = LAY != QR_LAYOUT_PAPER;
    if (mode == kModeRank4 || mode == kModePrefix) {
        if constexpr (LAY == QR_LAYOUT_INLINE32X2) {
            return nullptr;  // sigma 2 only
        } else {
            if (mode == kModeRank4)
                return n32 && kN32 ? region_rank<LAY, true, false, 2, 4, 1, 16, true, kModeRank4, false, kN32>
                                   : region_rank<LAY, true, false, 2, 4, 1, 16, true, kModeRank4>;
            return n32 && kN32 ? region_rank<LAY, true, false, 2, 4, 1, 16, true, kModePrefix, false, kN32>
                               : region_rank<LAY, true, false, 2, 4, 1, 16, true, kModePrefix>;
        }
    }
    if (quad) {
        if constexpr (LAY == QR_LAYOUT_INLINE32X2) {
            return nullptr;
        } else {
            if (n32 && kN32) return vec ? pick_variant<LAY, true, true, kN32>(v) : pick_variant<LAY, true, false, kN32>(v);
            return vec ? pick_variant<LAY, true, true>(v) : pick_variant<LAY, true, false>(v);
        }
    }
    if constexpr (LAY == QR_LAYOUT_INLINE24_8) {
        return nullptr;  // sigma 4 only
    } else {
        if (n32 && kN32)
            return vec ? pick_variant<LAY, false, true, kN32>(v) : pick_variant<LAY, false, false, kN32>(v);
        return vec ? pick_variant<LAY, false, true>(v) : pick_variant<LAY, false, false>(v);
    }
}

RankFn pick_region_rank(int layout, bool quad, bool vec, int v, int mode, bool n32) {
    switch (layout) {
        case QR_LAYOUT_PAPER: return pick_rank_lay<QR_LAYOUT_PAPER>(quad, vec, v, mode, false);
        case QR_LAYOUT_SECTOR: return pick_rank_lay<QR_LAYOUT_SECTOR>(quad, vec, v, mode, n32);
        case QR_LAYOUT_INLINE32: return pick_rank_lay<QR_LAYOUT_INLINE32>(quad, vec, v, mode, n32);
        case QR_LAYOUT_INLINE32X2: return pick_rank_lay<QR_LAYOUT_INLINE32X2>(quad, vec, v, mode, n32);
        case QR_LAYOUT_INLINE24_8: return pick_rank_lay<QR_LAYOUT_INLINE24_8>(quad, vec, v, mode, n32);
        default: return nullptr;
    }
}

template <int LAY>
BaseFn pick_base_lay(bool quad, bool prefix, bool n32) {
    constexpr bool kN32 = LAY != QR_LAYOUT_PAPER;
    if constexpr (LAY == QR_LAYOUT_INLINE32X2) {
        if (quad || prefix) return nullptr;
    } else {
        if (prefix) return n32 && kN32 ? region_base<LAY, true, true, kN32> : region_base<LAY, true, true, false>;
        if (quad) return n32 && kN32 ? region_base<LAY, true, false, kN32> : region_base<LAY, true, false, false>;
    }
    if constexpr (LAY == QR_LAYOUT_INLINE24_8) {
        return nullptr;  // sigma 4 only
    } else {
        return n32 && kN32 ? region_base<LAY, false, false, kN32> : region_base<LAY, false, false, false>;
    }
}

BaseFn pick_region_base(int layout, bool quad, bool prefix, bool n32) {
    switch (layout) {
        case QR_LAYOUT_PAPER: return pick_base_lay<QR_LAYOUT_PAPER>(quad, prefix, false);
        case QR_LAYOUT_SECTOR: return pick_base_lay<QR_LAYOUT_SECTOR>(quad, prefix, n32);
        case QR_LAYOUT_INLINE32: return pick_base_lay<QR_LAYOUT_INLINE32>(quad, prefix, n32);
        case QR_LAYOUT_INLINE32X2: return pick_base_lay<QR_LAYOUT_INLINE32X2>(quad, prefix, n32);
        case QR_LAYOUT_INLINE24_8: return pick_base_lay<QR_LAYOUT_INLINE24_8>(quad, prefix, n32);
        default: return nullptr;
    }
}

int region_shift(uint64_t n) {
    int shift = 0;
    while ((n >> shift) >= kRegions) shift++;
    return shift;
}

// Regions in use.  The rank pass keeps about 2.4 regions in flight per 2^28
// queries (its ~4900 resident warps over the 2^11 steps of 16 runs that one
// region of a 2^28-query batch holds; fewer queries, proportionally more).
// Longer regions give longer runs per tile, which every pass pays for per
// run, until the lines in flight outgrow what the L2 keeps: measured on the
// full workloads, regions of up to 22 MB of index at 2^28 queries gained and
// 36 MB lost badly.  So the shift grows by one when the doubled region stays
// within 24 MiB of index per 2^28 queries of the batch.  Returns the extra
// shift (0 or 1).
int region_extra(const qr_index* idx, int shift, uint64_t m) {
    if (shift >= kMaxShift) return 0;
    const double bytes = (double)line_bytes(idx->layout) * (double)idx->nblocks;
    const double doubled = bytes * std::ldexp(1.0, shift + 1) / ((double)idx->n + 1.0);
    return doubled * std::ldexp(1.0, 28) <= (double)(24u << 20) * (double)m ? 1 : 0;
}

}  // namespace

bool region_supported(const qr_index* idx, int rank4) {
    // rank, rank_c, prefix_rank (sigma 4) and rank_4 (sigma 4) on the paper
    // and sector layouts, for texts whose regions fit the 29-bit key
    // (n < 2^37); chains and the 128-byte line layout run direct
    if (idx->layout == QR_LAYOUT_LINE128) return false;
    if (region_shift(idx->n) > kMaxShift) return false;
    return rank4 == 0 || idx->sigma == 4;
}

bool region_auto(const qr_index* idx, uint64_t m) {
    if (m < (1ull << 20) || m >= (1ull << 32)) return false;
    const uint64_t bytes = line_bytes(idx->layout) * idx->nblocks;
    const uint64_t l2 = (uint64_t)device_props().l2_bytes;
    // an index that fits comfortably in L2 gains nothing; a batch with fewer
    // than two queries per 128-byte DRAM line of the index has too little
    // reuse to pay for moving the queries
    return bytes > l2 / 2 && m * 64 >= bytes;
}

int launch_rank_regions(const qr_index* idx, const uint64_t* q, const uint8_t* cvec, int c, uint64_t m, uint64_t* out,
                        int rank4, cudaStream_t s, cudaEvent_t* marks, const DirectLaunch* direct) {
    if (m == 0) return QR_OK;
    if (m >= (1ull << 32)) return fail(QR_EINVAL, "region batch: m must be below 2^32");
    const int shift0 = region_shift(idx->n);
    if (shift0 > kMaxShift) return fail(QR_EINVAL, "region batch: n must be below 2^37");
    const int extra = region_extra(idx, shift0, m);
    const int shift = shift0 + extra;
    // regions that can hold valid queries (q <= n); out-of-range ones fall in the
    // last region and are never answered
    const uint64_t used = (idx->n >> shift) + 1 < kRegions ? (idx->n >> shift) + 1 : kRegions;
    const int mode = rank4 == 1 ? kModeRank4 : rank4 == 2 ? kModePrefix : kModeRank;
    const uint64_t tiles = (m + kTile - 1) / kTile;
    const uint64_t nseg = (uint64_t)kRegions * tiles;
    cudaMemPool_t pool;
    int rc = region_pool(&pool);
    if (rc) return rc;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    // the segment table twice: region-major (the rank pass walks it) and
    // tile-major (the unsort reads one tile's entries in one coalesced load)
    const size_t key_bytes = up(m * 4), idx_bytes = up(m * 2), seg_bytes = up(nseg * 4);
    const size_t res_bytes = mode == kModeRank4 ? up(m * 16) : 0;  // rank_4: the four counts' low 32 bits
    const size_t base_bytes = (size_t)kRegions * kBaseSyms * 8;
    void* buf = nullptr;
    // under stream capture the scratch becomes a graph memory node
    // (cudaMallocAsync); otherwise it comes from the library's pool
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "region batch: capture status");
    const size_t scratch = key_bytes + idx_bytes + 2 * seg_bytes + base_bytes + res_bytes + 32;
    e = cap == cudaStreamCaptureStatusActive ? cudaMallocAsync(&buf, scratch, s)
                                             : cudaMallocFromPoolAsync(&buf, scratch, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(QR_ENOMEM, "region batch: no scratch memory");
    }
    char* cur = (char*)buf;
    uint32_t* keys = (uint32_t*)cur;
    uint16_t* idxs = (uint16_t*)(cur += key_bytes);
    uint32_t* seg = (uint32_t*)(cur += idx_bytes);
    uint32_t* segt = (uint32_t*)(cur += seg_bytes);
    uint64_t* bases = (uint64_t*)(cur += seg_bytes);
    uint32_t* res16 = (uint32_t*)(cur += base_bytes);
    unsigned long long* counters = (unsigned long long*)(cur + res_bytes);  // queue, probe, abort
    static std::once_flag once[64];
    static int once_rc[64];
    const int dev = device_props().device & 63;
    std::call_once(once[dev], [&] {
        once_rc[dev] = set_smem(region_sort<false>, kSortSmem);
        if (!once_rc[dev]) once_rc[dev] = set_smem(region_sort<true>, kSortSmem);
        if (!once_rc[dev]) once_rc[dev] = set_smem(region_sort_tma<false>, kSortTmaSmem);
        if (!once_rc[dev]) once_rc[dev] = set_smem(region_sort_tma<true>, kSortTmaSmem);
        if (!once_rc[dev]) once_rc[dev] = set_smem(region_unsort, kUnsortSmem);
        if (!once_rc[dev]) once_rc[dev] = set_smem(region_unsort4, kUnsort4Smem);
    });
    rc = once_rc[dev];
    const bool quad = idx->sigma == 4, vec = cvec != nullptr;
    const bool n32 = idx->layout != QR_LAYOUT_PAPER && idx->n < (1ull << 37);
    const int sms = device_props().sms;
    Gate gate{nullptr, 0, counters + 2};
    if (!rc) {
        e = cudaMemsetAsync(counters, 0, 24, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "region batch: counter reset");
    }
    if (!rc && direct) {
        // probe, then the direct kernels: they run only for a clustered batch
        const uint64_t probes = tiles < (uint64_t)kProbeTiles ? tiles : (uint64_t)kProbeTiles;
        region_probe<<<(unsigned)probes, 256, 0, s>>>(q, m, shift, tiles, counters + 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "region_probe");
        gate = Gate{counters + 1, (unsigned long long)probes * kClusterMax, counters + 2};
        if (!rc) rc = (*direct)(gate.count, gate.limit);
    }
    if (!rc) {
        // the bases the unsort pass restores the results from
        BaseFn bf = pick_region_base(idx->layout, quad, mode == kModePrefix, n32);
        if (!bf) {
            rc = fail(QR_EINVAL, "region batch: no base kernel for this layout and call");
        } else {
            bf<<<kRegions * kBaseSyms / 256, 256, 0, s>>>(idx->lines, idx->supers, idx->n, shift, bases, gate);
            e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_fail(e, "region_base");
        }
    }
    if (!rc && marks) cudaEventRecord(marks[0], s);
    if (!rc) {
        const uint64_t grid = tiles < (uint64_t)sms * kPassBlocks ? tiles : (uint64_t)sms * kPassBlocks;
        // the bulk copies need 16-byte aligned query and symbol arrays (the
        // key and index arrays are)
        const bool tma = (((uintptr_t)q | (uintptr_t)cvec) & 15) == 0;
        if (tma) {
            const uint64_t g1 = tiles < (uint64_t)sms ? tiles : (uint64_t)sms;
            auto sort_fn = vec ? region_sort_tma<true> : region_sort_tma<false>;
            sort_fn<<<(unsigned)g1, kTmaThreads, kSortTmaSmem, s>>>(q, vec ? cvec : nullptr, (uint32_t)c,
                                                                     (uint32_t)idx->sigma, m, idx->n, shift, tiles,
                                                                     keys, idxs, seg, segt, idx->status, gate,
                                                                     idx->region_withhold);
        } else {
            auto sort_fn = vec ? region_sort<true> : region_sort<false>;
            sort_fn<<<(unsigned)grid, kPassThreads, kSortSmem, s>>>(q, vec ? cvec : nullptr, (uint32_t)c,
                                                                    (uint32_t)idx->sigma, m, idx->n, shift, tiles,
                                                                    keys, idxs, seg, segt, idx->status, gate);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "region_sort");
    }
    if (!rc && marks) cudaEventRecord(marks[1], s);
    if (!rc) {
        RankFn fn = pick_region_rank(idx->layout, quad, vec, idx->region_variant, mode, n32);
        if (!fn) {
            cudaFreeAsync(buf, s);
            return fail(QR_EINVAL, "region batch: no rank pass for this layout and call");
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRankThreads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        // the segment table is region-major: the runs of the regions in use
        // come first (out-of-range queries, in the last region, are never
        // answered)
        const uint64_t nseg_used = used * tiles;
        const uint64_t nsteps = (nseg_used + 7) / 8;
        const uint64_t need = (nsteps + kRankThreads / 32 - 1) / (kRankThreads / 32);
        uint64_t grid = (uint64_t)per_sm * sms;
        if (grid > need) grid = need;
        RankPassArgs ra;
        ra.keys = keys;
        ra.res16 = res16;
        ra.seg = seg;
        ra.nseg = nseg_used;
        ra.tiles = tiles;
        ra.lines = idx->lines;
        ra.supers = idx->supers;
        ra.c0 = (uint32_t)c;
        ra.shift = shift;
        ra.queue = counters;
        ra.gate = gate;
        fn<<<(unsigned)grid, kRankThreads, 0, s>>>(ra);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "region_rank");
    }
    if (!rc && marks) cudaEventRecord(marks[2], s);
    if (!rc && mode != kModeRank4) {
        const uint64_t grid = tiles < (uint64_t)sms * 2 ? tiles : (uint64_t)sms * 2;
        region_unsort<<<(unsigned)grid, kUnsortThreads, kUnsortSmem, s>>>(keys, idxs, segt, bases, m, tiles,
                                                                          (uint32_t)used, out, gate);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "region_unsort");
    }
    if (!rc && mode == kModeRank4) {
        const uint64_t grid = tiles < (uint64_t)sms ? tiles : (uint64_t)sms;
        region_unsort4<<<(unsigned)grid, kUnsort4Threads, kUnsort4Smem, s>>>(
            res16, idxs, segt, bases, m, tiles, (uint32_t)used, out, ((uintptr_t)out & 31) == 0, gate);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "region_unsort4");
    }
    if (!rc && marks) cudaEventRecord(marks[3], s);
    cudaFreeAsync(buf, s);
    return rc;
}

int region_trim() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& p : g_pool)
        if (p) QR_CUDA_TRY(cudaMemPoolTrimTo(p, 0));
    return QR_OK;
}

}  // namespace qr
