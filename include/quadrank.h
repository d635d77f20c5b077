/*
 * quadrank.h -- C ABI of libquadrank.so: batched rank queries over BiRank
 * (binary alphabet) and QuadRank (2-bit DNA alphabet) in the cache-line
 * interleaved, delta-to-the-middle layout, and the QuadFm count-only
 * backward search built on QuadRank, on one NVIDIA GB300 (sm_103a).
 *
 * Source of the operations: R. Groot Koerkamp, "QuadRank: Engineering a High
 * Throughput Rank", arXiv 2602.04103 (cited below as "the paper").
 *
 * Conventions shared by every entry point
 *   - Return value: QR_OK (0) or one of the QR_E* codes below; the message of
 *     the last failure on the calling host thread is qr_last_error().
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Query calls only enqueue work on it and return; their device
 *     buffers must stay valid until the stream reaches that point.
 *   - "device pointer" arguments are caller-owned CUDA device (or managed)
 *     memory; the library never frees them.  Index memory allocated by a
 *     *_build call is owned by the returned handle and released by *_free.
 *   - Errors found on the device while a query runs (a position q > n, a
 *     pattern byte > 3) do not fail the call: they write the documented
 *     sentinel output and set a bit in the handle's device status word,
 *     which qr_status / qfm_status read (synchronising) and clear.
 *   - A handle may be used from one host thread at a time; concurrent query
 *     calls on different streams with the same handle are allowed.
 *
 * Text formats
 *   bit text (sigma = 2): bit i = (text[i / 64] >> (i % 64)) & 1.
 *   DNA text (sigma = 4): char i = (text[i / 32] >> (2 * (i % 32))) & 3 with
 *                         A = 0, C = 1, G = 2, T = 3.
 *   DNA codes           : one byte per char, values 0..3.
 *   Bits / chars at positions >= n inside the last word are ignored.
 */
#ifndef QUADRANK_H
#define QUADRANK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QR_OK 0
#define QR_EINVAL 1    /* bad argument (size, sigma, symbol, null pointer)        */
#define QR_ENOMEM 2    /* a device or pinned-host allocation failed              */
#define QR_ECUDA 3     /* a CUDA runtime call failed (message in qr_last_error)  */
#define QR_ERANGE 4    /* status bit: some query had q > n                        */
#define QR_ETIMEOUT 16 /* status bit: a bounded device wait gave up               */
#define QR_EBADSYM 8   /* status bit: some pattern byte was > 3                   */

#define QR_LAYOUT_PAPER 0   /* BiRank16 / QuadRank16 exactly as in the paper      */
#define QR_LAYOUT_LINE128 2 /* one 128-byte line per query (the GPU's DRAM fill   */
                            /* unit), read by 4 lanes in one instruction: sigma 2 */
                            /* = 16-bit delta + 1008 bits (1.69%), sigma 4 = four */
                            /* deltas + 480 transposed chars (6.88%), deltas to   */
                            /* the line middle                                     */
#define QR_LAYOUT_SECTOR 1  /* one self-contained 32-byte sector per query:       */
                            /* sigma 2 = the paper's BiRank16x2 (two 16-bit deltas */
                            /* at 1/4 and 3/4 of a 480-bit block, 6.72%), each     */
                            /* delta at the head of its 32-byte half; sigma 4 =    */
                            /* four deltas + 96 transposed chars per sector (33%)  */
#define QR_LAYOUT_INLINE32 3    /* 32-bit inline values (paper Sec. 3.1 BiRank32,   */
                                /* Sec. 4.1 QuadRank32): sigma 2 = one 32-bit value */
                                /* + 480 data bits per line (6.67%), the value to   */
                                /* data offset 240; sigma 4 = four 32-bit values +  */
                                /* 192 transposed chars (33.3%), values to char 96; */
                                /* a query reads the whole 64-byte line              */
#define QR_LAYOUT_INLINE32X2 4  /* sigma 2 only: the paper's BiRank32x2 (Sec. 3.1),  */
                                /* two 32-bit values, each at the head of its        */
                                /* 32-byte half with 224 data bits, pointing to the  */
                                /* half's middle (14.3%); one sector per query       */
#define QR_LAYOUT_INLINE24_8 5  /* sigma 4 only: the paper's QuadRank24_8 (Sec.    */
                                /* 4.1), 192 transposed chars in 3 groups of 64,   */
                                /* per symbol a 24-bit value to the end of group 0 */
                                /* and an 8-bit step from there to the end of      */
                                /* group 2: a query counts at most 64 chars (33.3%) */
/* The inline layouts have no superblock array of 32-bit offsets: their
 * values are relative to an L0 table of one 64-bit rank per 2^22 lines (2^16
 * for QR_LAYOUT_INLINE24_8; four ranks for sigma 4), which shrinks it by a
 * factor 2^15 (2^9) against the 16-bit layouts (a few KB at n = 2^43), as the
 * paper's variants intend. */

typedef struct qr_index qr_index;

/* Sizes of a built rank index. */
typedef struct {
    uint64_t n;             /* text length (bits or chars)                           */
    int32_t sigma;          /* 2 or 4                                                */
    int32_t layout;         /* QR_LAYOUT_*                                           */
    uint64_t block_chars;   /* chars per line: 496 / 224 (paper layout), 480 / 192   */
                            /* (sector), 1008 / 480 (128-byte lines), 480 / 192      */
                            /* (inline 32), 448 (inline 32 x2) for sigma 2 / 4       */
    uint64_t super_blocks;  /* lines per superblock: 128 / 256 (paper, sector),      */
                            /* 32 / 64 (128-byte lines) for sigma 2 / 4; 2^22 lines  */
                            /* per L0 entry (inline layouts)                         */
    uint64_t line_bytes;    /* 64, or 128 for QR_LAYOUT_LINE128                      */
    uint64_t nblocks;       /* floor(n / B) + 1 lines                                */
    uint64_t nsuper;        /* ceil(nblocks / super_blocks) superblock entries        */
    uint64_t bytes_blocks;  /* line_bytes * nblocks                                  */
    uint64_t bytes_super;   /* 4 * nsuper (sigma 2) or 16 * nsuper (sigma 4); inline */
                            /* layouts 8 * nsuper or 32 * nsuper                     */
} qr_info_t;

/* Per-handle launch tuning of the rank kernels (chosen by the autotuner). */
typedef struct {
    int32_t queries_per_thread;  /* independent queries in flight per thread: 1,2,4,8 */
                                 /* (1 or 2 for QR_LAYOUT_LINE128)                   */
    int32_t block_threads;       /* 64..512, multiple of 32                            */
    int32_t load_mode;           /* 0: whole 64-byte line, 16-byte loads;               */
                                 /* 1: only the 32-byte sectors the query needs, 16-byte */
                                 /*    loads; 2: whole line, 32-byte loads; 3: needed    */
                                 /*    sectors, 32-byte loads; 4: whole line, the two    */
                                 /*    lanes of a pair load its two sectors in one       */
                                 /*    instruction (one request per line)                */
                                 /* The sector and inline layouts ignore it (one      */
                                 /* 32-byte load; whole lines by lane pairs).          */
    int32_t grid_blocks;         /* 0: SM count x resident blocks per SM                */
} qr_tuning_t;

/* Message of the last failure on this host thread ("" if none). */
const char* qr_last_error(void);

/* ABI version of this header (bumped on any signature change). */
int qr_abi_version(void);

/*
 * qr_build -- build the rank index of a packed text.
 * Paper: Sec. 3 (BiRank16: 16-bit delta b_j inlined in each 64-byte line,
 * B = 496 data bits per block, S = 128 B, shifted 32-bit superblock offsets
 * s_i = floor(rank(iS) / 2^11), b_j = rank(jB + 240) - 2^11 s_{j/128}; parallel
 * construction: per-superblock counts, a prefix sum, then independent
 * superblocks) and Sec. 4 (QuadRank16: four 16-bit deltas b_{j,c} to the
 * middle of each block, B4 = 224 chars, S4 = 256 B4, s_{i,c} =
 * floor(rank(iS4, c) / 2^13), transposed negated low/high bit words).
 *   text           packed text (format above), ceil(n/64) (sigma 2) or ceil(n/32)
 *                  (sigma 4) uint64 words; host memory if text_on_device == 0,
 *                  device memory otherwise.  Only read during the call.
 *   n              text length; n < 2^43 (sigma 2) or n < 2^45 (sigma 4).
 *   sigma          2 or 4.
 *   stream         stream the build runs on; the call returns after the build
 *                  has completed (it synchronises the stream).
 *   out            receives the handle (owner: caller, release with qr_free).
 * Errors: QR_EINVAL (sigma, n out of range, null pointers), QR_ENOMEM, QR_ECUDA.
 */
int qr_build(const uint64_t* text, uint64_t n, int sigma, int text_on_device, void* stream, qr_index** out);

/* qr_build with an explicit layout (QR_LAYOUT_*).  QR_LAYOUT_SECTOR follows the
 * paper's BiRank16x2 variant (Sec. 3.1: two 16-bit deltas, to 1/4 and 3/4 of
 * the block, so only a quarter of the line is popcounted); the sigma 4 form
 * applies the same idea to QuadRank (Sec. 4.1 variants: larger inline values
 * so that fewer characters are counted).  Every query reads one 32-byte
 * sector of its line.  QR_LAYOUT_INLINE32 and QR_LAYOUT_INLINE32X2 are the
 * paper's 32-bit inline variants (Sec. 3.1 BiRank32 and BiRank32x2, Sec. 4.1
 * QuadRank32) and QuadRank24_8 (Sec. 4.1, QR_LAYOUT_INLINE24_8).
 * QR_LAYOUT_INLINE32X2 with sigma 4 and QR_LAYOUT_INLINE24_8 with sigma 2
 * give QR_EINVAL. */
int qr_build_ex(const uint64_t* text, uint64_t n, int sigma, int text_on_device, int layout, void* stream,
                qr_index** out);

/*
 * qr_rank -- out[k] = rank(q[k], c) for k < m, one symbol c for all queries.
 * Paper: Sec. 1 (definition rank(q, c) = #{i < q : t_i = c}, 0 <= q <= n),
 * Sec. 3 Eq. (1) (BiRank: 2^11 s_{i_q} + b_{j_q} plus or minus the popcount of
 * at most 256 bits between q and the block middle), Sec. 4 "rank1" and the
 * App. A listing (QuadRank: 2^13 s_{i,c} + b_{j,c} plus or minus at most 128
 * chars matched as (lo ^ cl) & (hi ^ ch)).  For sigma 2, c = 1 is rank(q) and
 * c = 0 is q - rank(q).
 *   q, out  device pointers to m uint64 values each (may not overlap).
 *   c       0..sigma-1.
 * A query with q > n yields out[k] = UINT64_MAX and sets QR_ERANGE in the status.
 * Errors (returned): QR_EINVAL (null index/pointers with m > 0, c out of range),
 * QR_ECUDA (launch failure).  m = 0 is a no-op.
 */
int qr_rank(const qr_index* idx, const uint64_t* q, uint64_t m, int c, uint64_t* out, void* stream);

/*
 * qr_rank_c -- out[k] = rank(q[k], c[k]): one symbol per query.
 * Paper: as qr_rank.  c is a device array of m bytes, each in 0..sigma-1; a
 * byte >= sigma yields UINT64_MAX and sets QR_EBADSYM in the status.
 */
int qr_rank_c(const qr_index* idx, const uint64_t* q, const uint8_t* c, uint64_t m, uint64_t* out, void* stream);

/*
 * qr_rank4 -- out4[4k + c] = rank(q[k], c) for c = 0..3 (sigma 4 only).
 * Paper: Sec. 4 "4-way popcount" (rank_4: all four counts of one line; the
 * sign of (q mod B) - 96 decides add or subtract).
 *   out4  device pointer to 4 m uint64 values, row-major (query-major).
 * q > n yields four UINT64_MAX and QR_ERANGE.  Errors: QR_EINVAL (sigma != 4).
 */
int qr_rank4(const qr_index* idx, const uint64_t* q, uint64_t m, uint64_t* out4, void* stream);

/*
 * qr_prefix_rank -- out[k] = rank(q[k], 0) + ... + rank(q[k], c): the number
 * of characters at most c before q[k] (sigma 4 only), the operation the paper
 * names for a bidirectional FM-index (Sec. 6, future work); computed from the
 * same line as rank_4.  c in 0..3; q > n gives UINT64_MAX and QR_ERANGE.
 * Errors: QR_EINVAL (sigma != 4, c out of range, NULL buffers with m > 0).
 */
int qr_prefix_rank(const qr_index* idx, const uint64_t* q, uint64_t m, int c, uint64_t* out, void* stream);

/*
 * qr_rank_chain -- dependent queries (the paper's latency measurement, Sec.
 * 5.1: each query depends on the result of the previous one).  Chain k starts
 * at q0[k] and takes `steps` queries:
 *   r_t = rank(q_t, c),  q_{t+1} = floor(x (n + 1) / 2^64)  with
 *   x = (q_t + r_t) * 0x9E3779B97F4A7C15 mod 2^64,
 * so a chain has one line in flight at a time; chains run in parallel, one
 * per thread, and every layout reads one line (one request) per query.
 * out2[2k] = q_{steps-1} (the last position queried), out2[2k+1] =
 * r_{steps-1}.  A start q0[k] > n gives two UINT64_MAX and QR_ERANGE.
 * Errors: QR_EINVAL (steps = 0, c out of range, NULL buffers), QR_ECUDA.
 */
int qr_rank_chain(const qr_index* idx, const uint64_t* q0, uint64_t nchains, uint64_t steps, int c, uint64_t* out2,
                  void* stream);

/*
 * qr_rank_host / qr_rank4_host -- the same queries with HOST buffers: the
 * call streams q to the device in chunks, runs the kernel and copies the
 * results back, overlapping the three on internal streams, and returns when
 * out (or out4) holds every result.  q and out should be pinned (page-locked)
 * host memory for full copy bandwidth; pageable memory works but is slower.
 * c < 0 means per-query symbols in c_host (m bytes); otherwise c is the symbol.
 * Device staging buffers are allocated on first use and kept by the handle.
 * Errors: as qr_rank, plus QR_ENOMEM for the staging buffers.
 */
int qr_rank_host(qr_index* idx, const uint64_t* q_host, const uint8_t* c_host, uint64_t m, int c,
                 uint64_t* out_host, void* stream);
int qr_rank4_host(qr_index* idx, const uint64_t* q_host, uint64_t m, uint64_t* out4_host, void* stream);

/* Sizes of the index.  Errors: QR_EINVAL on null arguments. */
int qr_info(const qr_index* idx, qr_info_t* info);

/* Device pointers of the 64-byte lines and of the superblock array (for
 * inspection of the layout; owned by the handle). */
int qr_layout_ptrs(const qr_index* idx, const void** lines, const void** supers);

/* Copy the layout out for inspection: lines_dst receives bytes_blocks bytes,
 * supers_dst bytes_super bytes (either may be NULL; host or device memory).
 * Synchronises stream.  Errors: QR_EINVAL, QR_ECUDA. */
int qr_copy_layout(const qr_index* idx, void* lines_dst, void* supers_dst, void* stream);

/* Read the launch tuning / set it (values are validated; QR_EINVAL if not). */
int qr_get_tuning(const qr_index* idx, qr_tuning_t* t);
int qr_set_tuning(qr_index* idx, const qr_tuning_t* t);

/*
 * qr_autotune -- time the rank kernel of this index for every supported
 * tuning (queries in flight per thread 1/2/4/8, block of 128/256/512 threads,
 * every load mode of the layout) on the caller's queries, keep the fastest in
 * the handle and return it in *best (may be NULL).  Timing: CUDA events on
 * `stream`, best of 3 launches per candidate after one warm-up.
 *   q        device queries (m of them, m >= 1); they should look like the
 *            production batch (same size class and distribution).
 *   mode     0: qr_rank with symbol c; 1: qr_rank_c with c_vec; 2: qr_rank4.
 *   out      device scratch output: m uint64 (4 m for mode 2).
 * The candidates run the direct kernels (region batching, where the handle
 * would use it, is switched off while they are timed).
 * Synchronises stream.  Errors: QR_EINVAL, QR_ECUDA.  This library's own
 * addition: the paper tunes by hand per CPU (Sec. 3.1 and 4.1 variants).
 */
int qr_autotune(qr_index* idx, const uint64_t* q, uint64_t m, int mode, int c, const uint8_t* c_vec, uint64_t* out,
                void* stream, qr_tuning_t* best);

/*
 * qr_build_tuned -- build the index in every layout whose space overhead is at
 * most max_overhead (fraction of the text size, e.g. 0.10), autotune each as
 * qr_autotune does on the first min(m, 2^24) of the given queries, time each
 * tuned index on all m queries (by the path qr_rank takes for a batch of m,
 * region batching included) and return the fastest; the others are freed.
 * *layout_out (may be NULL) receives the chosen QR_LAYOUT_*.
 * Overheads: sigma 2 paper 3.28%, sector 6.72%, 128-byte lines 1.69%; sigma 4
 * paper 14.40%, sector 33.46%, 128-byte lines 6.88%.
 * Errors: QR_EINVAL (no layout within max_overhead), as qr_build.
 */
int qr_build_tuned(const uint64_t* text, uint64_t n, int sigma, int text_on_device, double max_overhead,
                   const uint64_t* q, uint64_t m, int mode, int c, const uint8_t* c_vec, uint64_t* out, void* stream,
                   qr_index** idx_out, int* layout_out);

/*
 * Region batching -- how qr_rank and qr_rank_c answer a large batch.
 * The paper answers each query from its own cache line and hides the
 * latency of the line by prefetching while it works through a batch of
 * independent queries (Sec. 3 "Prefetching", Sec. 5.1 for-loop and prefetch
 * modes).  On GB300 a random 64-byte line costs a whole 128-byte DRAM fill,
 * so a batch that holds several queries per line of the index is answered
 * faster by moving the queries instead: the batch is cut into tiles of 8192
 * queries, every tile is sorted by text region in shared memory (at most
 * 256 regions, region = q >> shift; the shift grows by one for an index that
 * is small against the batch, so that regions hold more queries), the sorted
 * runs are answered region after region (the lines of the regions in flight
 * stay in L2, each line is read from DRAM about once per batch) and every
 * tile's results are put back in query order.  Every result is computed by the same query arithmetic from
 * the same line, so the outputs are those of the direct kernels, bit for
 * bit.  This is this library's own addition; the paper has no counterpart.
 *   QR_BATCH_AUTO     (default) region batching when the index is not
 *                     L2-resident (more than half of L2), 2^20 <= m < 2^32 and
 *                     the batch holds at least two queries per 128 bytes of
 *                     index; the direct kernels otherwise.  When region
 *                     batching is chosen, a probe kernel first counts the
 *                     regions met by the leading 1024 queries of 64 tiles; a
 *                     clustered batch (at most 4 regions per probe on
 *                     average, e.g. sorted queries, whose neighbours share
 *                     lines) is answered by the direct kernels instead.  The
 *                     choice is made on the device: both paths are launched
 *                     and the one not chosen returns at once.
 *   QR_BATCH_DIRECT   always the direct kernels (one line load per query).
 *   QR_BATCH_REGIONS  region batching for every m < 2^32 (larger batches
 *                     run direct).
 * Scope: qr_rank, qr_rank_c, qr_prefix_rank and qr_rank4 on the paper and
 * sector layouts, for n < 2^37 (a position inside its region must fit 29
 * bits); chains, the 128-byte line layout and larger texts run direct.
 * Between the passes a query keeps 4 bytes of result (rank_4: 16), the low
 * 32 bits of each count, restored from the count at the first position of
 * its region.
 * Scratch: 6 bytes per query (a 4-byte key and a 2-byte index inside the
 * tile; rank_4 16 more), 8 bytes per (region, tile) pair (1/4 byte per
 * query), an 8 KiB table of region bases and 32 bytes of counters (work
 * queue, probe count, abort word), from a memory pool of the library that
 * keeps the memory for later calls (released by qr_release_scratch).  When
 * that memory cannot be had, the call runs the direct kernels instead.
 * Status bits and sentinel outputs are those of the direct kernels.
 */
#define QR_BATCH_AUTO 0
#define QR_BATCH_DIRECT 1
#define QR_BATCH_REGIONS 2

/* Set the batch mode of the handle (QR_BATCH_*).  Errors: QR_EINVAL. */
int qr_set_batch_mode(qr_index* idx, int mode);

/* *plan = the path a call of m queries would take on this handle:
 * QR_BATCH_DIRECT or QR_BATCH_REGIONS (rank4: 0 rank / rank_c, 1 rank_4,
 * 2 prefix_rank).  Under QR_BATCH_AUTO, QR_BATCH_REGIONS means region
 * batching subject to the device-side probe for clustered batches.
 * Errors: QR_EINVAL (NULL arguments, rank4 out of range). */
int qr_rank_plan(const qr_index* idx, uint64_t m, int rank4, int* plan);

/* Measurement aid: with enable != 0, region-batched calls on this handle
 * record CUDA events between their three passes (sort, rank, unsort).  With
 * ms3 != NULL the call first waits for the last such call and writes the
 * three pass durations in milliseconds.  Not for concurrent calls on one
 * handle.  Errors: QR_EINVAL (ms3 before timing was enabled), QR_ECUDA. */
int qr_region_timing(qr_index* idx, int enable, float* ms3);

/* Launch tuning of the rank pass of region batching: variant 0..3 =
 * (items in flight per lane, resident blocks of 256 threads per SM, rounds
 * of work items loaded ahead) of (2, 4, 1) (default), (1, 6, 2), (2, 4, 1)
 * with the index lines loaded under an L2 evict-last policy, (4, 3, 1).
 * Errors: QR_EINVAL. */
int qr_set_region_tuning(qr_index* idx, int variant);

/* Test hook of the failure path: with withhold != 0, the first block of the
 * sort pass never issues its first bulk copy, so its bounded wait (0.25 s)
 * runs out.  The call then sets QR_ETIMEOUT in the status, its rank and
 * unsort passes return without touching out, and the context stays usable
 * for the next call.  It only applies when the TMA sort runs (aligned query,
 * symbol and work arrays with at least one full tile).  Errors: QR_EINVAL. */
int qr_set_region_fault(qr_index* idx, int withhold);

/* Return the pooled scratch memory of region batching to the device (on every
 * device the library has used).  Errors: QR_ECUDA. */
int qr_release_scratch(void);

/* Synchronise stream, return the OR of the status bits (QR_ERANGE, QR_EBADSYM,
 * QR_ETIMEOUT; each >= 4) set by queries since the last call, and clear them;
 * 0 when all were valid.  A failure of the call itself returns QR_EINVAL or
 * QR_ECUDA (both < 4). */
int qr_status(qr_index* idx, void* stream);

/* Release the index (waits for the device to finish using it). NULL is a no-op. */
int qr_free(qr_index* idx);

/*
 * qr_probe_gather -- measurement aid: out[k] = XOR of the `bytes`-byte record
 * at a random record index of buf for m draws, read with load_bytes-byte (16
 * or 32) vector loads, with the same threads-and-loads-in-flight scheme as the
 * rank kernels.  load_bytes = 128 (records of 128 bytes only) reads each
 * record as the 128-byte line layout's rank kernels read a line: the four
 * lanes of a quad each load one 32-byte sector of it in the same instruction.
 * It gives the random-access ceiling of this GPU's memory for records of 32,
 * 64 or 128 bytes, the GPU counterpart of the paper's measured random-access
 * limit of RAM (Sec. 5.1, "Lower bounds": 2.5 ns per cache line in total).
 *   buf    device buffer of nrec * bytes bytes, 16-byte aligned.
 *   seed   splitmix64 seed of the record indices (uniform in [0, nrec)).
 *   out    device array of m uint64 (one digest per draw, defeats dead-code
 *          elimination).
 * Errors: QR_EINVAL (bytes not 16/32/64/128, load_bytes not 16/32/128 or 128
 * with bytes != 128, nrec = 0, no kernel for
 * (bytes, queries_per_thread) -- 128-byte records allow at most 4 in flight).
 */
int qr_probe_gather(const void* buf, uint64_t nrec, int bytes, int load_bytes, uint64_t m, uint64_t seed,
                    uint64_t* out, int queries_per_thread, int block_threads, void* stream);

/*
 * qr_probe_l2 -- measurement aid: the rate of random 64-byte record reads
 * (two 32-byte vector loads each) from a buffer small enough to stay in L2,
 * the memory the QuadFm count kernel reads its index from (App. D: an index
 * of 2^26 characters is about 20 MB).  It gives the count kernel's ceiling,
 * as qr_probe_gather gives the HBM ceiling of the rank kernels (Sec. 5.1,
 * "Lower bounds").
 *   buf       device buffer of nrec * 64 bytes, 32-byte aligned (the first
 *             call brings it into L2; time the calls after it).
 *   mode      0: each thread reads 4 independent records per round (the L2
 *             random-read throughput); 1: each thread runs one chain, a
 *             round reads 2 records whose indices depend on the previous
 *             round's data, as the two interval ends of an LF step depend
 *             on the step before.
 *   nthreads  threads in all (one digest each); rounds >= 1 per thread.
 *             Records read: 4 * nthreads * rounds (mode 0) or
 *             2 * nthreads * rounds (mode 1).
 *   seed      splitmix64 seed of the record indices (uniform in [0, nrec)).
 *   out       device array of nthreads uint64 (digests).
 * Errors: QR_EINVAL (mode, nrec = 0 or above 2^40, buf unaligned, rounds = 0,
 * block_threads not 64..256 and a multiple of 32).
 */
int qr_probe_l2(const void* buf, uint64_t nrec, int mode, uint64_t nthreads, uint32_t rounds, uint64_t seed,
                uint64_t* out, int block_threads, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QUADRANK_H */
