/*
 * quadfm.h -- C ABI of the QuadFm count-only FM-index in libquadrank.so:
 * index construction over a DNA text and batched exact-match counting by
 * backward search over a QuadRank16 structure holding the BWT.
 *
 * Source: R. Groot Koerkamp, "QuadRank: Engineering a High Throughput Rank",
 * arXiv 2602.04103, App. D ("QuadFm: A Batching FM-index").  Conventions
 * (return codes, streams, ownership, status bits) are those of quadrank.h.
 */
#ifndef QUADFM_H
#define QUADFM_H

#include "quadrank.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qfm_index qfm_index;


typedef struct {
    uint64_t n;            /* text length (chars); the BWT has n + 1 rows     */
    uint64_t dollar_row;   /* BWT row of the sentinel $                       */
    uint64_t C[5];         /* C[c] = 1 + #chars < c; C[4] = n + 1             */
    uint64_t bytes_rank;   /* bytes of the QuadRank16 structure over the BWT  */
    uint64_t bytes_table;  /* bytes of the 8-mer table                        */
    int32_t kmer;          /* prefix-table length (8)                          */
    int32_t has_sa;        /* 1 if the suffix array was kept (QFM_KEEP_SA)     */
    int32_t sa_sample;     /* suffix-array sampling factor for locate (0: none) */
    int32_t reserved;
    uint64_t bytes_locate; /* bytes of the locate structures (marks + samples) */
} qfm_info_t;

#define QFM_KEEP_SA 1      /* qfm_build flag: keep the suffix array for export */

/*
 * qfm_build -- build the count-only FM-index of a DNA text.
 * Paper: App. D (QuadFm: one sentinel $ whose BWT position is stored, the
 * BWT held in a QuadRank16 structure, an 8-character prefix lookup table that
 * replaces the first 8 search steps).  The paper does not describe suffix
 * array construction; this library sorts the suffixes of T$ by prefix
 * doubling on the GPU.
 *   codes  n bytes 0..3 (host if codes_on_device == 0, else device).
 *   n      1 <= n < 2^32 - 1.
 *   flags  0 or QFM_KEEP_SA.
 *   stream the call synchronises it before returning.
 * Errors: QR_EINVAL (n, null, a byte > 3), QR_ENOMEM, QR_ECUDA.
 */
int qfm_build(const uint8_t* codes, uint64_t n, int codes_on_device, int flags, void* stream, qfm_index** out);

/*
 * qfm_count_approx -- out[k] = number of text positions where pattern k
 * matches with at most max_mismatches substituted characters (Hamming
 * distance), by backtracking backward search.  Paper: Sec. 1 (rank_4, all
 * four ranks of a position at once, serves approximate pattern matching in an
 * FM-index), Sec. 4 rank_4, App. D backward search.  Every node of the search
 * extends its interval by all four characters from rank_4 of both ends; the
 * prefix table is not used (a mismatch may fall in the last 8 characters).
 * One persistent launch with a device work queue, as qfm_count.
 *   max_mismatches  0..3 (0 gives the exact counts of qfm_count, and runs
 *                   its kernel).
 * The empty pattern counts n + 1.  A pattern holding a byte > 3 anywhere, or
 * with out-of-order offsets, yields 0 and sets QR_EBADSYM.  The work grows
 * with the number of strings within the distance that occur in T: about
 * (3 |P|)^k nodes near the start of a search over a random text.
 * Errors: QR_EINVAL (NULL with m > 0, max_mismatches out of range),
 * QR_ENOMEM, QR_ECUDA.
 */
int qfm_count_approx(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, int max_mismatches,
                     uint64_t* out, void* stream);

/*
 * qfm_build_ex -- qfm_build that also prepares locate queries when
 * sa_sample > 0.  The paper names locate as the natural extension of its
 * FM-index (Sec. 6) without a method; its comparison indexes sample the
 * suffix array (App. D results, "suffix-array sampling factor").  Here the
 * rows whose suffix starts at a multiple of sa_sample are marked in a
 * BiRank16 index over the n + 1 rows (Sec. 3), and the sampled positions
 * divided by sa_sample are stored in row order: (n + 1) / 8 * 1.033 +
 * 4 (n / sa_sample + 1) bytes on top of the count index.  A locate then takes
 * at most sa_sample - 1 LF steps per occurrence.
 *   sa_sample  0 (count only) or >= 1.  Other arguments as qfm_build.
 * Errors: as qfm_build.
 */
int qfm_build_ex(const uint8_t* codes, uint64_t n, int codes_on_device, int flags, uint32_t sa_sample, void* stream,
                 qfm_index** out);

/*
 * qfm_locate -- the text positions of every occurrence of m patterns.
 * Paper: Sec. 6 (locate, future work); the search is App. D's backward search
 * (the persistent count kernel, which also records each pattern's
 * suffix-array interval [lo, hi)); each row of an interval is then walked by
 * LF steps to a sampled row: SA[r] = sa_sample * sample + steps.
 *   patterns, offsets  as qfm_count.
 *   occ        device array of m + 1 uint64: occ[k] = index in `positions` of
 *              pattern k's first occurrence, occ[m] = total (the exclusive
 *              scan of the counts).
 *   positions  device array of `capacity` uint64, or NULL to only compute occ
 *              and *total.  positions[occ[k] .. occ[k+1]) are pattern k's
 *              occurrences in suffix-array row order (the order of the
 *              suffixes starting there; sort them for text order).
 *   total      host pointer: receives the number of occurrences.
 * The call synchronises the stream once (to read the total) and returns with
 * the locate kernel queued on it.  Patterns with a byte > 3 or out-of-order
 * offsets have no occurrences and set QR_EBADSYM in the status; the empty
 * pattern occurs at 0..n.  Scratch: 16 m + 16 bytes from the stream-ordered
 * pool of the stream.
 * Errors: QR_EINVAL (NULL arguments, index built without a sampling factor),
 * QR_ERANGE (positions given and total > capacity: occ and *total are valid,
 * positions untouched), QR_ENOMEM, QR_ECUDA.
 */
int qfm_locate(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* occ,
               uint64_t* positions, uint64_t capacity, uint64_t* total, void* stream);

/*
 * qfm_count -- out[k] = number of occurrences of pattern k in T, for k < m,
 * in one persistent kernel: every warp pulls pattern ids from a device work
 * queue (an atomic counter), each lane runs one backward search (8-mer table,
 * then LF steps lo = C[c] + rank(lo, c) - [c = 0 and lo > dollar_row], same for
 * hi, while lo < hi), and a lane whose search ends is refilled at once.
 * Paper: App. D (query_batch: a batch of active searches, finished ones
 * swapped out, rank + LF for the rest), Sec. 4 rank1.
 *   patterns  device bytes 0..3, pattern k = patterns[offsets[k] .. offsets[k+1]);
 *             the whole range [patterns, patterns + offsets[m]) must be readable
 *             (the kernel reads it in aligned 16-byte chunks inside that range).
 *   offsets   device array of m + 1 non-decreasing uint64.
 *   out       device array of m uint64.
 * The empty pattern counts n + 1 (every position 0..n).  A pattern holding a
 * byte > 3, or whose offsets are out of order (offsets[k+1] < offsets[k] or
 * beyond offsets[m]), yields 0 and sets QR_EBADSYM in the status.  The call allocates a
 * 16-byte work-queue counter from the stream-ordered pool of the stream.
 * Errors: QR_EINVAL (null with m > 0), QR_ENOMEM, QR_ECUDA.
 */
int qfm_count(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* out,
              void* stream);

/*
 * qfm_count_ex -- qfm_count with flags.  QFM_BOTH_STRANDS also counts the
 * reverse complement of every pattern (A<->T, C<->G, reversed), as the paper's
 * QuadFm benchmark counts each read in both directions (App. D): out then
 * holds 2 m counts, out[k] for pattern k and out[m + k] for its reverse
 * complement, all from the same persistent launch (the reverse complement is
 * read from the pattern bytes on the fly).  Other arguments and errors as
 * qfm_count; unknown flags give QR_EINVAL.
 */
#define QFM_BOTH_STRANDS 2
int qfm_count_ex(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* out,
                 int flags, void* stream);

/*
 * qfm_count_stepwise -- the same counts with one kernel launch per search step
 * (the plain form: a table-lookup launch, then launches that each advance
 * every active search by one character).  Kept as the comparison baseline.
 * It allocates per-pattern state (24 bytes x m) from the stream-ordered pool
 * and synchronises the stream once to learn the longest pattern.
 */
int qfm_count_stepwise(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m,
                       uint64_t* out, void* stream);

/*
 * qfm_count_noalloc -- qfm_count that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they count -- code that runs inside a memory pool or
 * allocator owned by another framework, under a hard device-memory budget,
 * or on a latency path where an allocation call is not allowed.
 * Same arguments, results and status bits as qfm_count; the caller still
 * passes every input and output buffer.  The kernel's only scratch, its
 * work-queue counter (16 bytes, for any m), lives in a static 256-byte
 * device array of the library instead of the stream-ordered pool; every GPU
 * that loads the library holds that array until the process exits.  A call
 * whose scratch need exceeded the array would be rejected with QR_EINVAL
 * (the need is fixed, so valid calls are never rejected).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  All calls share the one array
 * and reset its counter at the start: calls whose executions overlap on the
 * GPU (different streams, no ordering between them) race on it and must not
 * be issued; calls ordered on one stream are fine.
 * Errors: QR_EINVAL (null arguments with m > 0), QR_ECUDA.
 */
int qfm_count_noalloc(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m,
                      uint64_t* out, void* stream);

/* L2 policy of the persistent count kernel: 0 = plain read-only loads;
 * 1 = index lines and superblock entries loaded evict-last and the pattern /
 * offset stream evict-first; 2 (default) = index evict-last, patterns and
 * offsets under the default policy.  The index stays L2-resident under 1 and
 * 2; under 1 a pattern's 32-byte sector was often evicted between the two
 * 16-byte halves its search reads and fetched twice (measured, 10^7
 * patterns over 2^26 characters: 1.60 GB of DRAM reads per launch under 1,
 * 0.95 GB under 2, 3.4 GB under 0).  Errors: QR_EINVAL. */
int qfm_set_policy(qfm_index* idx, int policy);

/* Index facts.  Errors: QR_EINVAL. */
int qfm_info(const qfm_index* idx, qfm_info_t* info);

/* Copy the index pieces to caller device buffers (any pointer may be NULL):
 * sa (n + 1 uint32, requires QFM_KEEP_SA), bwt codes (n + 1 bytes, the $ row
 * holds 0), table (4^8 x 2 uint64: [lo, hi) of every 8-mer, k-mer index
 * sum code_i 4^(7-i)).  Synchronises stream. */
int qfm_export(const qfm_index* idx, uint32_t* sa, uint8_t* bwt, uint64_t* table, void* stream);

/* The rank index over the BWT (owned by the FM index). */
const qr_index* qfm_rank_index(const qfm_index* idx);

/* As qr_status, for the FM index. */
int qfm_status(qfm_index* idx, void* stream);

/* Release (waits for the device). NULL is a no-op. */
int qfm_free(qfm_index* idx);

/* ---------------------------------------------------------------------- */
/* Continuous-batching server over one index                               */
/* ---------------------------------------------------------------------- */
/*
 * The paper processes reads in batches inside each thread (App. D); this
 * server is the host runtime that turns a stream of independent count
 * requests into such batches on the GPU.  A worker thread owns `slots` batch
 * slots (device buffers carved from budget_bytes, pinned staging, a stream).
 * Whenever a slot is free and requests wait, it packs waiting requests in
 * arrival order while they fit (max_batch_patterns, max_batch_bytes,
 * max_requests_per_batch), runs qfm_count on the slot's stream and copies the
 * counts back, so requests that arrive while earlier batches run are admitted
 * into the next free slot and their work overlaps on the device.  Completion
 * is polled from the host (no device-side waits).  With slots = 1 and
 * max_requests_per_batch = 1 the server is the plain per-request path.
 */
typedef struct qfm_server qfm_server;

typedef struct {
    uint64_t budget_bytes;          /* device memory for all slots                     */
    int32_t slots;                  /* batches in flight (1..64)                        */
    int32_t max_requests_per_batch; /* >= 1                                             */
    uint64_t max_batch_patterns;    /* patterns per batch (a request may not exceed it) */
    uint64_t max_batch_bytes;       /* pattern bytes per batch (same)                   */
    int32_t poll_us;                /* worker's completion-poll interval                */
    int32_t fail_after_batches;     /* test hook: > 0 makes batch k+1 fail on the host  */
    int32_t use_graph;              /* 1: each batch is one launch of the slot's CUDA   */
                                    /*    graph (copy in, reset queue, count, copy out) */
                                    /*    with updated node parameters; 0: stream calls */
    int32_t reserved;
} qfm_server_opts_t;

typedef struct {
    uint64_t submitted, completed, pending, in_flight, batches;
    double mean_requests_per_batch;
    int32_t error;                  /* first error of the server (QR_OK if none)        */
    int32_t reserved;
    uint64_t graph_batches;         /* batches launched as one CUDA graph                */
} qfm_server_stats_t;

/* Fill *opts with defaults: 1 GiB budget, 4 slots, 2^20 patterns and 64 MiB
 * of pattern bytes per batch, no limit on requests per batch, 20 us poll,
 * batches launched as CUDA graphs. */
int qfm_server_default_opts(qfm_server_opts_t* opts);

/* Start a server (allocates the slots; the index must outlive it).
 * Errors: QR_EINVAL (options, slots x capacity above the budget), QR_ENOMEM. */
int qfm_server_create(qfm_index* idx, const qfm_server_opts_t* opts, qfm_server** out);

/* Queue one request of m >= 1 patterns (host memory, pattern k =
 * patterns[offsets[k] .. offsets[k+1])); counts go to out[0..m) (host).  The
 * buffers must stay untouched until the request completes.  Returns at once.
 * When consecutive requests of a batch lie back to back in the same pinned
 * buffers (patterns, offsets and out), the batch is copied straight from and
 * to them; otherwise through the slot's pinned staging.  Malformed offsets
 * give count 0 and QR_EBADSYM (see qfm_count).
 * Errors: QR_EINVAL (NULL, offsets[m] < offsets[0], larger than a slot). */
int qfm_server_submit(qfm_server* sv, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* out,
                      uint64_t* request_id);

/* Take up to cap completed requests: ids, latency (submit to completion, us)
 * and status (QR_OK or the error that failed the request); *n_done = count. */
int qfm_server_poll(qfm_server* sv, uint64_t* ids, double* latency_us, int* status, uint64_t cap, uint64_t* n_done);

/* Wait until every submitted request has completed (QR_ETIMEOUT after
 * timeout_s seconds); returns the server's error if a batch failed. */
int qfm_server_drain(qfm_server* sv, double timeout_s);

int qfm_server_stats(qfm_server* sv, qfm_server_stats_t* stats);

/* Stop after the queued requests complete, free the slots. NULL is a no-op. */
int qfm_server_destroy(qfm_server* sv);

/* Replay a request trace from a native thread: request r (patterns
 * req_first[r] .. req_first[r+1] of the pattern set `offsets`) is submitted
 * arrival_s[r] seconds after the start; the call waits for all, writes counts
 * to out (indexed like the pattern set), per-request latency_us[r] and the
 * makespan.  The server must have no other submitters or unpolled requests. */
int qfm_server_replay(qfm_server* sv, const uint8_t* patterns, const uint64_t* offsets, const uint64_t* req_first,
                      uint64_t nreq, const double* arrival_s, uint64_t* out, double* latency_us, double* makespan_s);

#ifdef __cplusplus
}
#endif
#endif /* QUADFM_H */
