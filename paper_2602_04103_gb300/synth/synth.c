/*
 * Seeded synthetic inputs for the rank and FM-count workloads.
 *
 * This module only draws data: packed bit texts, packed DNA texts, query
 * positions, query symbols, an FM text with planted repeats and a pattern
 * set.  It contains none of the rank or backward-search arithmetic, and it is
 * the one piece of code that both the CPU oracle (tests) and the CUDA path
 * (tests, benchmark) consume, so that both sides see byte-identical inputs.
 *
 * Randomness: a counter-based splitmix64 (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014; finaliser
 * constants as published with Vigna's reference implementation).  Value i of
 * stream s is mix(s + (i + 1) * golden_gamma).  Everything is a pure function
 * of (seed, index), so any slice can be regenerated independently and in
 * parallel.
 *
 * Formats (shared with the C-ABI):
 *   bit text  : bit i = (words[i / 64] >> (i % 64)) & 1, bits >= n are 0.
 *   DNA text  : char i = (words[i / 32] >> (2 * (i % 32))) & 3, A=0 C=1 G=2 T=3,
 *               chars >= n are 0.
 *   DNA codes : one byte per char, values 0..3.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Value i of the stream with the given seed. */
uint64_t qs_splitmix64(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * GOLDEN_GAMMA); }

/* Seed of sub-stream k of a base seed (text, queries, symbols, ...). */
uint64_t qs_substream(uint64_t seed, uint64_t k) { return qs_splitmix64(seed ^ 0xD1B54A32D192ED03ULL, k); }

/* floor(x * r / 2^64): maps a uniform 64-bit draw to [0, r). */
static inline uint64_t mulhi_range(uint64_t x, uint64_t r) { return (uint64_t)(((unsigned __int128)x * r) >> 64); }

/* Threshold t such that P(draw < t) = p for a uniform 64-bit draw. */
static uint64_t prob_threshold(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return UINT64_MAX;
    return (uint64_t)(p * 18446744073709551616.0);
}

/* ---- a small parallel-for over [0, total) ---- */
typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } range_job;

static void* range_thread(void* arg) {
    range_job* j = (range_job*)arg;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static int g_threads = 0;

int qs_set_threads(int t) { g_threads = t; return 0; }

int qs_threads(void) {
    if (g_threads > 0) return g_threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

static void parallel_for(uint64_t total, range_fn fn, void* ctx) {
    int t = qs_threads();
    if (total < 4096 || t == 1) { fn(ctx, 0, total); return; }
    if ((uint64_t)t > total) t = (int)total;
    pthread_t th[64];
    range_job jobs[64];
    uint64_t chunk = (total + t - 1) / t;
    int started = 0;
    for (int k = 0; k < t; k++) {
        uint64_t lo = chunk * k, hi = lo + chunk;
        if (lo >= total) break;
        if (hi > total) hi = total;
        jobs[k].fn = fn; jobs[k].ctx = ctx; jobs[k].lo = lo; jobs[k].hi = hi;
        if (pthread_create(&th[k], NULL, range_thread, &jobs[k]) != 0) {
            fn(ctx, lo, hi);           /* no thread available: run inline */
            jobs[k].fn = NULL;
        }
        started = k + 1;
    }
    for (int k = 0; k < started; k++)
        if (jobs[k].fn) pthread_join(th[k], NULL);
}

/* ---- bit texts ---- */
typedef struct { uint64_t seed, n, thr; int half; uint64_t* words; } bits_ctx;

static void bits_range(void* vc, uint64_t lo, uint64_t hi) {
    bits_ctx* c = (bits_ctx*)vc;
    for (uint64_t w = lo; w < hi; w++) {
        uint64_t v = 0;
        if (c->half) {
            v = qs_splitmix64(c->seed, w);
        } else {
            uint64_t base = w * 64;
            for (int b = 0; b < 64; b++)
                v |= (uint64_t)(qs_splitmix64(c->seed, base + b) < c->thr) << b;
        }
        uint64_t first = w * 64;
        if (first + 64 > c->n) {
            uint64_t keep = c->n > first ? c->n - first : 0;
            v = keep == 0 ? 0 : (v & (keep == 64 ? ~0ULL : ((1ULL << keep) - 1)));
        }
        c->words[w] = v;
    }
}

/* i.i.d. bits with P(1) = p, packed LSB-first into ceil(n/64) words.
 * p == 0.5 draws one 64-bit value per word; other p draw one value per bit. */
int qs_bits(uint64_t seed, uint64_t n, double p, uint64_t* words) {
    bits_ctx c = {seed, n, prob_threshold(p), p == 0.5, words};
    parallel_for((n + 63) / 64, bits_range, &c);
    return 0;
}

/* ---- DNA texts ---- */
typedef struct { uint64_t seed, n; uint64_t* words; } dna_ctx;

static void dna_range(void* vc, uint64_t lo, uint64_t hi) {
    dna_ctx* c = (dna_ctx*)vc;
    for (uint64_t w = lo; w < hi; w++) {
        uint64_t v = qs_splitmix64(c->seed, w);
        uint64_t first = w * 32;
        if (first + 32 > c->n) {
            uint64_t keep = c->n > first ? c->n - first : 0;
            v = keep == 0 ? 0 : (v & ((1ULL << (2 * keep)) - 1));
        }
        c->words[w] = v;
    }
}

/* i.i.d. uniform {A,C,G,T}, 2-bit packed into ceil(n/32) words (one draw = 32 chars). */
int qs_dna_uniform(uint64_t seed, uint64_t n, uint64_t* words) {
    dna_ctx c = {seed, n, words};
    parallel_for((n + 31) / 32, dna_range, &c);
    return 0;
}

typedef struct { uint64_t seed, n, tA, tC, tG; uint64_t* words; } gc_ctx;

static void gc_range(void* vc, uint64_t lo, uint64_t hi) {
    gc_ctx* c = (gc_ctx*)vc;
    for (uint64_t w = lo; w < hi; w++) {
        uint64_t v = 0;
        for (int k = 0; k < 32; k++) {
            uint64_t i = w * 32 + k;
            if (i >= c->n) break;
            uint64_t x = qs_splitmix64(c->seed, i);
            uint64_t code = x < c->tA ? 0 : x < c->tC ? 1 : x < c->tG ? 2 : 3;
            v |= code << (2 * k);
        }
        c->words[w] = v;
    }
}

static inline void set_code(uint64_t* words, uint64_t i, uint64_t code) {
    uint64_t sh = 2 * (i % 32);
    words[i / 32] = (words[i / 32] & ~(3ULL << sh)) | (code << sh);
}

/* DNA with GC content gc (P(C)=P(G)=gc/2, P(A)=P(T)=(1-gc)/2), then homopolymer
 * runs: run r has a uniform start, a uniform length in [run_min, run_max] and a
 * uniform symbol, and runs are written until their lengths (clipped to the text)
 * add up to at least run_cover * n.  Packed 2-bit. */
int qs_dna_gc_runs(uint64_t seed, uint64_t n, double gc, double run_cover, uint64_t run_min,
                   uint64_t run_max, uint64_t* words) {
    double pa = (1.0 - gc) / 2.0, pc = gc / 2.0;
    gc_ctx c = {qs_substream(seed, 1), n, prob_threshold(pa), prob_threshold(pa + pc),
                prob_threshold(pa + 2 * pc), words};
    parallel_for((n + 31) / 32, gc_range, &c);
    if (n == 0 || run_cover <= 0.0) return 0;
    uint64_t rs = qs_substream(seed, 2);
    uint64_t target = (uint64_t)(run_cover * (double)n), covered = 0;
    for (uint64_t r = 0; covered < target; r++) {
        uint64_t start = mulhi_range(qs_splitmix64(rs, 3 * r), n);
        uint64_t len = run_min + mulhi_range(qs_splitmix64(rs, 3 * r + 1), run_max - run_min + 1);
        uint64_t sym = qs_splitmix64(rs, 3 * r + 2) & 3;
        if (start + len > n) len = n - start;
        for (uint64_t i = start; i < start + len; i++) set_code(words, i, sym);
        covered += len;
    }
    return 0;
}

/* ---- queries and symbols ---- */
typedef struct { uint64_t seed, range; uint64_t* q; } q_ctx;

static void q_range(void* vc, uint64_t lo, uint64_t hi) {
    q_ctx* c = (q_ctx*)vc;
    for (uint64_t i = lo; i < hi; i++) c->q[i] = mulhi_range(qs_splitmix64(c->seed, i), c->range);
}

/* m positions uniform in [0, n] (inclusive). */
int qs_queries(uint64_t seed, uint64_t n, uint64_t m, uint64_t* q) {
    q_ctx c = {seed, n + 1, q};
    parallel_for(m, q_range, &c);
    return 0;
}

typedef struct { uint64_t seed, mask; uint8_t* c; } s_ctx;

static void s_range(void* vc, uint64_t lo, uint64_t hi) {
    s_ctx* c = (s_ctx*)vc;
    for (uint64_t i = lo; i < hi; i++) c->c[i] = (uint8_t)(qs_splitmix64(c->seed, i) & c->mask);
}

/* m symbols uniform in [0, sigma), sigma in {2, 4}. */
int qs_symbols(uint64_t seed, uint64_t m, int sigma, uint8_t* c) {
    if (sigma != 2 && sigma != 4) return 1;
    s_ctx ctx = {seed, (uint64_t)sigma - 1, c};
    parallel_for(m, s_range, &ctx);
    return 0;
}

/* ---- format conversions (2-bit packed <-> one byte per char) ---- */
typedef struct { const uint8_t* codes; uint64_t n; uint64_t* words; } pack_ctx;

static void pack_range(void* vc, uint64_t lo, uint64_t hi) {
    pack_ctx* c = (pack_ctx*)vc;
    for (uint64_t w = lo; w < hi; w++) {
        uint64_t v = 0;
        for (int k = 0; k < 32; k++) {
            uint64_t i = w * 32 + k;
            if (i >= c->n) break;
            v |= (uint64_t)(c->codes[i] & 3) << (2 * k);
        }
        c->words[w] = v;
    }
}

int qs_pack2(const uint8_t* codes, uint64_t n, uint64_t* words) {
    pack_ctx c = {codes, n, words};
    parallel_for((n + 31) / 32, pack_range, &c);
    return 0;
}

typedef struct { const uint64_t* words; uint64_t n; uint8_t* codes; } unpack_ctx;

static void unpack_range(void* vc, uint64_t lo, uint64_t hi) {
    unpack_ctx* c = (unpack_ctx*)vc;
    for (uint64_t i = lo; i < hi; i++) c->codes[i] = (uint8_t)((c->words[i / 32] >> (2 * (i % 32))) & 3);
}

int qs_unpack2(const uint64_t* words, uint64_t n, uint8_t* codes) {
    unpack_ctx c = {words, n, codes};
    parallel_for(n, unpack_range, &c);
    return 0;
}

/* ---- FM text with planted repeats ---- */
typedef struct { uint64_t seed, n; uint8_t* codes; } fmt_ctx;

static void fmt_range(void* vc, uint64_t lo, uint64_t hi) {
    fmt_ctx* c = (fmt_ctx*)vc;
    for (uint64_t i = lo; i < hi; i++)
        c->codes[i] = (uint8_t)((qs_splitmix64(c->seed, i / 32) >> (2 * (i % 32))) & 3);
}

/* i.i.d. uniform DNA (one byte per char), then planted repeats: repeat r copies a
 * segment of uniform length [len_min, len_max] from a uniform source to a uniform
 * destination, substituting each copied base with probability sub_rate by one of
 * the other three bases (uniformly), until the copied lengths add up to at least
 * repeat_cover * n.  Repeats are applied in order r = 0, 1, ... */
int qs_fm_text(uint64_t seed, uint64_t n, double repeat_cover, uint64_t len_min, uint64_t len_max,
               double sub_rate, uint8_t* codes) {
    fmt_ctx c = {qs_substream(seed, 1), n, codes};
    parallel_for(n, fmt_range, &c);
    if (n == 0 || repeat_cover <= 0.0) return 0;
    if (len_max > n) len_max = n;
    if (len_min > len_max) len_min = len_max;
    uint8_t* tmp = (uint8_t*)malloc(len_max ? len_max : 1);
    if (!tmp) return 2;
    uint64_t rs = qs_substream(seed, 2), ss = qs_substream(seed, 3);
    uint64_t thr = prob_threshold(sub_rate);
    uint64_t target = (uint64_t)(repeat_cover * (double)n), covered = 0, draw = 0;
    for (uint64_t r = 0; covered < target; r++) {
        uint64_t len = len_min + mulhi_range(qs_splitmix64(rs, 3 * r), len_max - len_min + 1);
        uint64_t src = mulhi_range(qs_splitmix64(rs, 3 * r + 1), n - len + 1);
        uint64_t dst = mulhi_range(qs_splitmix64(rs, 3 * r + 2), n - len + 1);
        memcpy(tmp, codes + src, len);
        for (uint64_t k = 0; k < len; k++, draw++) {
            uint64_t x = qs_splitmix64(ss, 2 * draw);
            if (x < thr) {
                uint64_t y = qs_splitmix64(ss, 2 * draw + 1);
                tmp[k] = (uint8_t)((tmp[k] + 1 + mulhi_range(y, 3)) & 3);
            }
        }
        memcpy(codes + dst, tmp, len);
        covered += len;
    }
    free(tmp);
    return 0;
}

/* ---- pattern sets ---- */

/* offsets[0..m]: pattern k has length uniform in [len_min, len_max]. Returns the total. */
uint64_t qs_pattern_offsets(uint64_t seed, uint64_t m, uint64_t len_min, uint64_t len_max, uint64_t* offsets) {
    uint64_t ls = qs_substream(seed, 4), acc = 0;
    offsets[0] = 0;
    for (uint64_t k = 0; k < m; k++) {
        acc += len_min + mulhi_range(qs_splitmix64(ls, k), len_max - len_min + 1);
        offsets[k + 1] = acc;
    }
    return acc;
}

typedef struct {
    uint64_t seed, n, thr;
    const uint8_t* text;
    const uint64_t* offsets;
    uint8_t* out;
} pat_ctx;

static void pat_range(void* vc, uint64_t lo, uint64_t hi) {
    pat_ctx* c = (pat_ctx*)vc;
    for (uint64_t k = lo; k < hi; k++) {
        uint64_t ks = qs_splitmix64(c->seed, k);
        uint64_t len = c->offsets[k + 1] - c->offsets[k];
        uint8_t* p = c->out + c->offsets[k];
        if ((k & 1) == 0 && len <= c->n) {
            /* sampled from the text at a uniform start, then substituted */
            uint64_t start = mulhi_range(qs_splitmix64(ks, 0), c->n - len + 1);
            for (uint64_t t = 0; t < len; t++) {
                uint8_t b = c->text[start + t];
                uint64_t x = qs_splitmix64(ks, 2 * t + 1);
                if (x < c->thr) b = (uint8_t)((b + 1 + mulhi_range(qs_splitmix64(ks, 2 * t + 2), 3)) & 3);
                p[t] = b;
            }
        } else {
            /* i.i.d. uniform */
            for (uint64_t t = 0; t < len; t++)
                p[t] = (uint8_t)((qs_splitmix64(ks, t / 32) >> (2 * (t % 32))) & 3);
        }
    }
}

/* Fill patterns (one byte per base) for the offsets above: even k is a substring of
 * text at a uniform start with per-base substitution probability sub_rate, odd k is
 * i.i.d. uniform. */
int qs_patterns(uint64_t seed, const uint8_t* text, uint64_t n, uint64_t m, const uint64_t* offsets,
                double sub_rate, uint8_t* out) {
    pat_ctx c = {qs_substream(seed, 5), n, prob_threshold(sub_rate), text, offsets, out};
    parallel_for(m, pat_range, &c);
    return 0;
}
