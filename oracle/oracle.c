/*
 * ORACLE -- test infrastructure, not part of the product.
 *
 * Plain, slow, obviously correct CPU definitions of what the CUDA path
 * computes.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  It shares no code, header, table or
 * constant with the CUDA path; it reads the same packed inputs (the C-ABI's
 * text formats) and nothing else.
 *
 * Definitions followed (QuadRank paper, arXiv 2602.04103):
 *   rank(q, c) = #{ i < q : t_i = c },  0 <= q <= n          (Sec. 1, rank definition)
 *   rank(q)    = rank(q, 1) for the binary alphabet          (Sec. 1, Sec. 3)
 *   rank_4(q)  = (rank(q,0), rank(q,1), rank(q,2), rank(q,3)) (Sec. 4, rank_4)
 *   count(P)   = number of positions i with T[i .. i+|P|) = P, the quantity a
 *                count-only FM-index returns (App. D); equivalently the size
 *                of the suffix-array interval of suffixes of T$ prefixed by P.
 *   count_k(P) = number of positions i with T[i .. i+|P|) differing from P in
 *                at most k characters (approximate matching with
 *                substitutions, the use of rank_4 the paper names, Sec. 1).
 *   locate(P)  = those positions i themselves (the locate query the paper
 *                names as an extension of its FM-index, Sec. 6); listed in
 *                increasing order, or in suffix-array order (the order of the
 *                rows of P's interval).
 * The suffix array is the textbook one: all suffixes of T$ sorted, with the
 * sentinel $ smaller than every symbol (App. D stores one sentinel).
 *
 * Formats: bit text  bit i = (w[i/64] >> (i%64)) & 1;
 *          DNA text  char i = (w[i/32] >> (2*(i%32))) & 3 (A=0,C=1,G=2,T=3);
 *          DNA codes one byte per char.
 *
 * Parity pins live in tests/test_oracle_*.py.  Every function is
 * single-threaded on purpose, except or_rank_sweep_mt: the same sweep cut into
 * text chunks that threads answer side by side (pinned equal to the
 * single-threaded sweep), used to time the oracle on all host cores.
 */
#define _GNU_SOURCE
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_EINVAL = 1, OR_ERANGE = 4, OR_ENOMEM = 2 };

/* Symbol t_i of a packed text. */
static uint64_t text_char(const uint64_t* text, int sigma, uint64_t i) {
    if (sigma == 2) return (text[i / 64] >> (i % 64)) & 1;
    return (text[i / 32] >> (2 * (i % 32))) & 3;
}

uint64_t or_char(const uint64_t* text, int sigma, uint64_t i) { return text_char(text, sigma, i); }

/* rank(q, c) by the definition: a loop over t_0 .. t_{q-1}. */
int or_rank_naive(const uint64_t* text, uint64_t n, int sigma, uint64_t q, int c, uint64_t* out) {
    if ((sigma != 2 && sigma != 4) || c < 0 || c >= sigma) return OR_EINVAL;
    if (q > n) return OR_ERANGE;
    uint64_t r = 0;
    for (uint64_t i = 0; i < q; i++) r += text_char(text, sigma, i) == (uint64_t)c;
    *out = r;
    return OR_OK;
}

typedef struct { uint64_t q, idx; } qpair;

static int cmp_qpair(const void* a, const void* b) {
    const qpair* x = (const qpair*)a;
    const qpair* y = (const qpair*)b;
    if (x->q != y->q) return x->q < y->q ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/*
 * Many queries by one sweep: sort the queries by position, then walk the text
 * once from position 0, keeping the number of occurrences of every symbol in
 * t_0 .. t_{pos-1}; each query is answered when pos reaches it.
 *
 * mode 0: out[k] = rank(q[k], c)              (scalar c; c_arr == NULL)
 * mode 1: out[k] = rank(q[k], c_arr[k])
 * mode 2: out[4k + c] = rank(q[k], c), c = 0..sigma-1   (rank_4 for sigma = 4)
 * mode 3: out[k] = #{ i < q[k] : t_i <= c }            (prefix_rank, Sec. 6)
 * Queries with q > n get UINT64_MAX and the call returns OR_ERANGE.
 */
int or_rank_sweep(const uint64_t* text, uint64_t n, int sigma, const uint64_t* q, uint64_t m,
                  int mode, int c, const uint8_t* c_arr, uint64_t* out) {
    if (sigma != 2 && sigma != 4) return OR_EINVAL;
    if ((mode == 0 || mode == 3) && (c < 0 || c >= sigma)) return OR_EINVAL;
    if (mode == 2 && sigma != 4) return OR_EINVAL;
    qpair* ord = (qpair*)malloc((m ? m : 1) * sizeof(qpair));
    if (!ord) return OR_ENOMEM;
    for (uint64_t k = 0; k < m; k++) { ord[k].q = q[k]; ord[k].idx = k; }
    qsort(ord, m, sizeof(qpair), cmp_qpair);
    int rc = OR_OK;
    uint64_t pos = 0, cnt[4] = {0, 0, 0, 0};
    for (uint64_t k = 0; k < m; k++) {
        uint64_t target = ord[k].q, idx = ord[k].idx;
        if (target > n) {
            rc = OR_ERANGE;
            if (mode == 2) { for (int s = 0; s < 4; s++) out[4 * idx + s] = UINT64_MAX; }
            else out[idx] = UINT64_MAX;
            continue;
        }
        while (pos < target) {
            if (sigma == 2 && pos % 64 == 0 && pos + 64 <= target) {
                /* 64 whole bits at once: the number of ones is their popcount */
                uint64_t ones = (uint64_t)__builtin_popcountll(text[pos / 64]);
                cnt[1] += ones;
                cnt[0] += 64 - ones;
                pos += 64;
            } else {
                cnt[text_char(text, sigma, pos)]++;
                pos++;
            }
        }
        if (mode == 0) out[idx] = cnt[c];
        else if (mode == 3) {
            uint64_t r = 0;
            for (int s = 0; s <= c; s++) r += cnt[s];
            out[idx] = r;
        } else if (mode == 1) {
            int cc = c_arr[idx];
            if (cc >= sigma) { out[idx] = UINT64_MAX; rc = OR_EINVAL; }
            else out[idx] = cnt[cc];
        } else {
            for (int s = 0; s < 4; s++) out[4 * idx + s] = cnt[s];
        }
    }
    free(ord);
    return rc;
}

/*
 * The sweep of or_rank_sweep on `threads` threads (same modes, arguments,
 * results and return codes).  The text is cut into `threads` chunks of equal
 * length (a multiple of 64 positions); a query q belongs to the chunk that
 * holds position q (q = n to the last one).  Each thread first counts the
 * symbols of its chunk; a serial prefix sum of those totals gives the counts
 * before every chunk; then each thread sorts its own chunk's queries and
 * sweeps its chunk from that prefix, answering them as in or_rank_sweep.
 */
typedef struct {
    const uint64_t* text;
    uint64_t n, a, b;       /* chunk [a, b) of the text */
    int sigma, mode, c;
    const uint8_t* c_arr;
    qpair* ord;             /* this chunk's queries */
    uint64_t nq;
    uint64_t base[4];       /* symbol counts before position a */
    uint64_t total[4];      /* symbol counts of the chunk (phase 1) */
    uint64_t* out;
    int rc;
} sweep_job;

/* Phase 1: the symbol counts of t_a .. t_{b-1}. */
static void* sweep_totals(void* arg) {
    sweep_job* j = (sweep_job*)arg;
    uint64_t cnt[4] = {0, 0, 0, 0};
    for (uint64_t pos = j->a; pos < j->b;) {
        if (j->sigma == 2 && pos % 64 == 0 && pos + 64 <= j->b) {
            uint64_t ones = (uint64_t)__builtin_popcountll(j->text[pos / 64]);
            cnt[1] += ones;
            cnt[0] += 64 - ones;
            pos += 64;
        } else {
            cnt[text_char(j->text, j->sigma, pos)]++;
            pos++;
        }
    }
    memcpy(j->total, cnt, sizeof cnt);
    return NULL;
}

/* Phase 2: sort the chunk's queries and answer them by one sweep from a. */
static void* sweep_answer(void* arg) {
    sweep_job* j = (sweep_job*)arg;
    qsort(j->ord, j->nq, sizeof(qpair), cmp_qpair);
    uint64_t pos = j->a, cnt[4];
    memcpy(cnt, j->base, sizeof cnt);
    j->rc = OR_OK;
    for (uint64_t k = 0; k < j->nq; k++) {
        const uint64_t target = j->ord[k].q, idx = j->ord[k].idx;
        while (pos < target) {
            if (j->sigma == 2 && pos % 64 == 0 && pos + 64 <= target) {
                uint64_t ones = (uint64_t)__builtin_popcountll(j->text[pos / 64]);
                cnt[1] += ones;
                cnt[0] += 64 - ones;
                pos += 64;
            } else {
                cnt[text_char(j->text, j->sigma, pos)]++;
                pos++;
            }
        }
        if (j->mode == 0) j->out[idx] = cnt[j->c];
        else if (j->mode == 3) {
            uint64_t r = 0;
            for (int s = 0; s <= j->c; s++) r += cnt[s];
            j->out[idx] = r;
        } else if (j->mode == 1) {
            int cc = j->c_arr[idx];
            if (cc >= j->sigma) { j->out[idx] = UINT64_MAX; j->rc = OR_EINVAL; }
            else j->out[idx] = cnt[cc];
        } else {
            for (int s = 0; s < 4; s++) j->out[4 * idx + s] = cnt[s];
        }
    }
    return NULL;
}

int or_rank_sweep_mt(const uint64_t* text, uint64_t n, int sigma, const uint64_t* q, uint64_t m,
                     int mode, int c, const uint8_t* c_arr, uint64_t* out, int threads) {
    if (sigma != 2 && sigma != 4) return OR_EINVAL;
    if ((mode == 0 || mode == 3) && (c < 0 || c >= sigma)) return OR_EINVAL;
    if (mode == 2 && sigma != 4) return OR_EINVAL;
    if (mode < 0 || mode > 3 || threads < 1) return OR_EINVAL;
    const uint64_t T = (uint64_t)threads;
    uint64_t len = (n + T - 1) / T;
    len = (len + 63) / 64 * 64;
    if (len == 0) len = 64;
    sweep_job* jobs = (sweep_job*)calloc(T, sizeof(sweep_job));
    uint64_t* first = (uint64_t*)calloc(T + 1, sizeof(uint64_t));
    qpair* ord = (qpair*)malloc((m ? m : 1) * sizeof(qpair));
    pthread_t* tid = (pthread_t*)malloc(T * sizeof(pthread_t));
    if (!jobs || !first || !ord || !tid) {
        free(jobs); free(first); free(ord); free(tid);
        return OR_ENOMEM;
    }
    int rc = OR_OK;
    /* the chunk of every valid query; out-of-range queries are answered here */
    for (uint64_t k = 0; k < m; k++) {
        if (q[k] > n) continue;
        uint64_t ch = q[k] / len;
        if (ch >= T) ch = T - 1;
        first[ch + 1]++;
    }
    for (uint64_t t = 0; t < T; t++) first[t + 1] += first[t];
    uint64_t* fill = (uint64_t*)malloc(T * sizeof(uint64_t));
    if (!fill) {
        free(jobs); free(first); free(ord); free(tid);
        return OR_ENOMEM;
    }
    memcpy(fill, first, T * sizeof(uint64_t));
    for (uint64_t k = 0; k < m; k++) {
        if (q[k] > n) {
            rc = OR_ERANGE;
            if (mode == 2) { for (int s = 0; s < 4; s++) out[4 * k + s] = UINT64_MAX; }
            else out[k] = UINT64_MAX;
            continue;
        }
        uint64_t ch = q[k] / len;
        if (ch >= T) ch = T - 1;
        ord[fill[ch]].q = q[k];
        ord[fill[ch]].idx = k;
        fill[ch]++;
    }
    free(fill);
    for (uint64_t t = 0; t < T; t++) {
        sweep_job* j = &jobs[t];
        j->text = text; j->n = n; j->sigma = sigma; j->mode = mode; j->c = c; j->c_arr = c_arr; j->out = out;
        j->a = t * len < n ? t * len : n;
        j->b = (t + 1) * len < n ? (t + 1) * len : n;
        j->ord = ord + first[t];
        j->nq = first[t + 1] - first[t];
    }
    for (uint64_t t = 0; t < T; t++) pthread_create(&tid[t], NULL, sweep_totals, &jobs[t]);
    for (uint64_t t = 0; t < T; t++) pthread_join(tid[t], NULL);
    for (uint64_t t = 1; t < T; t++)
        for (int s = 0; s < 4; s++) jobs[t].base[s] = jobs[t - 1].base[s] + jobs[t - 1].total[s];
    for (uint64_t t = 0; t < T; t++) pthread_create(&tid[t], NULL, sweep_answer, &jobs[t]);
    for (uint64_t t = 0; t < T; t++) pthread_join(tid[t], NULL);
    for (uint64_t t = 0; t < T; t++)
        if (jobs[t].rc != OR_OK && rc == OR_OK) rc = jobs[t].rc;
    free(jobs); free(first); free(ord); free(tid);
    return rc;
}

/*
 * Dependent query chains (latency mode, Sec. 5.1): chain k starts at q0[k];
 * r_t = rank(q_t, c) and q_{t+1} = floor(x (n + 1) / 2^64) with
 * x = (q_t + r_t) * 0x9E3779B97F4A7C15 mod 2^64.  rank is read from a table
 * of prefix counts built by one pass over the text.  out[2k] = last position,
 * out[2k+1] = last rank.
 */
int or_rank_chain(const uint64_t* text, uint64_t n, int sigma, const uint64_t* q0, uint64_t nchains,
                  uint64_t steps, int c, uint64_t* out) {
    if ((sigma != 2 && sigma != 4) || c < 0 || c >= sigma || steps == 0) return OR_EINVAL;
    uint64_t* pref = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    if (!pref) return OR_ENOMEM;
    pref[0] = 0;
    for (uint64_t i = 0; i < n; i++) pref[i + 1] = pref[i] + (text_char(text, sigma, i) == (uint64_t)c);
    int rc = OR_OK;
    for (uint64_t k = 0; k < nchains; k++) {
        uint64_t q = q0[k], r = 0;
        if (q > n) {
            out[2 * k] = out[2 * k + 1] = UINT64_MAX;
            rc = OR_ERANGE;
            continue;
        }
        for (uint64_t t = 0; t < steps; t++) {
            r = pref[q];
            if (t + 1 < steps) {
                const uint64_t x = (q + r) * 0x9E3779B97F4A7C15ull;
                q = (uint64_t)(((unsigned __int128)x * (n + 1)) >> 64);
            }
        }
        out[2 * k] = q;
        out[2 * k + 1] = r;
    }
    free(pref);
    return rc;
}

/* ------------------------------------------------------------------ */
/* FM side: suffix array, BWT and occurrence counts by definition      */
/* ------------------------------------------------------------------ */

/* Compare suffixes i and j of T$ ($ = end of text, smaller than any symbol). */
static int cmp_suffix(const uint8_t* t, uint64_t n, uint64_t i, uint64_t j) {
    if (i == j) return 0;
    while (i < n && j < n) {
        if (t[i] != t[j]) return t[i] < t[j] ? -1 : 1;
        i++; j++;
    }
    /* one of them reached $: the one that ended is smaller */
    if (i == n) return -1;
    return 1;
}

typedef struct { const uint8_t* t; uint64_t n; } sa_ctx;

static int cmp_sa(const void* a, const void* b, void* arg) {
    const sa_ctx* c = (const sa_ctx*)arg;
    uint64_t i = *(const uint64_t*)a, j = *(const uint64_t*)b;
    return cmp_suffix(c->t, c->n, i, j);
}

/* sa[0 .. n] = the suffixes of T$ in lexicographic order (a comparison sort). */
int or_suffix_array(const uint8_t* codes, uint64_t n, uint64_t* sa) {
    for (uint64_t i = 0; i <= n; i++) sa[i] = i;
    sa_ctx c = {codes, n};
    qsort_r(sa, n + 1, sizeof(uint64_t), cmp_sa, &c);
    return OR_OK;
}

/* BWT of T$: bwt[k] = T[sa[k] - 1], and the row whose suffix is the whole text
 * holds $ -- reported as *dollar_row, with bwt[dollar_row] = 255. */
int or_bwt(const uint8_t* codes, uint64_t n, const uint64_t* sa, uint8_t* bwt, uint64_t* dollar_row) {
    for (uint64_t k = 0; k <= n; k++) {
        if (sa[k] == 0) { bwt[k] = 255; *dollar_row = k; }
        else bwt[k] = codes[sa[k] - 1];
    }
    return OR_OK;
}

/* Compare the first len chars of suffix s of T$ with pattern p:
 * < 0 if the suffix sorts before every string starting with p,
 * = 0 if the suffix starts with p, > 0 if it sorts after. */
static int cmp_prefix(const uint8_t* t, uint64_t n, uint64_t s, const uint8_t* p, uint64_t len) {
    for (uint64_t k = 0; k < len; k++) {
        if (s + k >= n) return -1;               /* reached $ first */
        if (t[s + k] != p[k]) return t[s + k] < p[k] ? -1 : 1;
    }
    return 0;
}

/* [lo, hi) = the rows of the suffix array whose suffixes start with p. */
int or_sa_interval(const uint8_t* codes, uint64_t n, const uint64_t* sa, const uint8_t* p, uint64_t len,
                   uint64_t* lo, uint64_t* hi) {
    uint64_t a = 0, b = n + 1;             /* first row with suffix >= p */
    while (a < b) {
        uint64_t mid = a + (b - a) / 2;
        if (cmp_prefix(codes, n, sa[mid], p, len) < 0) a = mid + 1; else b = mid;
    }
    uint64_t l = a;
    b = n + 1;                             /* first row with suffix > every extension of p */
    while (a < b) {
        uint64_t mid = a + (b - a) / 2;
        if (cmp_prefix(codes, n, sa[mid], p, len) <= 0) a = mid + 1; else b = mid;
    }
    *lo = l;
    *hi = a;
    return OR_OK;
}

/* count(P) by direct comparison at every start position (the empty pattern
 * occurs at each of the n + 1 positions 0..n). */
uint64_t or_count_brute(const uint8_t* codes, uint64_t n, const uint8_t* p, uint64_t len) {
    if (len == 0) return n + 1;
    if (len > n) return 0;
    uint64_t cnt = 0;
    for (uint64_t i = 0; i + len <= n; i++)
        if (codes[i] == p[0] && memcmp(codes + i, p, len) == 0) cnt++;
    return cnt;
}

/* Reverse complement of a DNA pattern: out[i] = 3 - p[len-1-i]
 * (A<->T, C<->G, read backwards), the other strand of the read (App. D). */
int or_revcomp(const uint8_t* p, uint64_t len, uint8_t* out) {
    for (uint64_t i = 0; i < len; i++) out[i] = (uint8_t)(3 - p[len - 1 - i]);
    return OR_OK;
}

/* count for m patterns (offsets[m+1]) via the suffix-array interval. */
int or_count_sa(const uint8_t* codes, uint64_t n, const uint64_t* sa, const uint8_t* pats,
                const uint64_t* offsets, uint64_t m, uint64_t* out) {
    for (uint64_t k = 0; k < m; k++) {
        uint64_t lo, hi;
        or_sa_interval(codes, n, sa, pats + offsets[k], offsets[k + 1] - offsets[k], &lo, &hi);
        out[k] = hi - lo;
    }
    return OR_OK;
}

/* locate for m patterns by direct comparison: occ[k] = index of pattern k's
 * first position in pos (occ[m] = total), positions in increasing order.  With
 * pos == NULL only occ is filled. */
int or_locate_brute(const uint8_t* codes, uint64_t n, const uint8_t* pats, const uint64_t* offsets, uint64_t m,
                    uint64_t* occ, uint64_t* pos) {
    uint64_t e = 0;
    for (uint64_t k = 0; k < m; k++) {
        const uint8_t* p = pats + offsets[k];
        const uint64_t len = offsets[k + 1] - offsets[k];
        occ[k] = e;
        for (uint64_t i = 0; i + len <= n; i++) {  /* the empty pattern: every i in 0..n */
            if (len == 0 || memcmp(codes + i, p, len) == 0) {
                if (pos) pos[e] = i;
                e++;
            }
        }
    }
    occ[m] = e;
    return OR_OK;
}

/* locate for m patterns via the suffix array: the positions sa[lo .. hi) of
 * each pattern's interval, in row order. */
int or_locate_sa(const uint8_t* codes, uint64_t n, const uint64_t* sa, const uint8_t* pats,
                 const uint64_t* offsets, uint64_t m, uint64_t* occ, uint64_t* pos) {
    uint64_t e = 0;
    for (uint64_t k = 0; k < m; k++) {
        uint64_t lo, hi;
        or_sa_interval(codes, n, sa, pats + offsets[k], offsets[k + 1] - offsets[k], &lo, &hi);
        occ[k] = e;
        for (uint64_t r = lo; r < hi; r++) {
            if (pos) pos[e] = sa[r];
            e++;
        }
    }
    occ[m] = e;
    return OR_OK;
}

/* count_k(P) by comparing P with every length-|P| window of T (the empty
 * pattern: every position 0..n, as count). */
uint64_t or_count_approx(const uint8_t* codes, uint64_t n, const uint8_t* p, uint64_t len, uint32_t k) {
    if (len == 0) return n + 1;
    if (len > n) return 0;
    uint64_t cnt = 0;
    for (uint64_t i = 0; i + len <= n; i++) {
        uint32_t d = 0;
        for (uint64_t j = 0; j < len && d <= k; j++) d += codes[i + j] != p[j];
        if (d <= k) cnt++;
    }
    return cnt;
}

int or_count_approx_batch(const uint8_t* codes, uint64_t n, const uint8_t* pats, const uint64_t* offsets,
                          uint64_t m, uint32_t k, uint64_t* out) {
    for (uint64_t j = 0; j < m; j++)
        out[j] = or_count_approx(codes, n, pats + offsets[j], offsets[j + 1] - offsets[j], k);
    return OR_OK;
}

/* count for m patterns by brute force. */
int or_count_brute_batch(const uint8_t* codes, uint64_t n, const uint8_t* pats, const uint64_t* offsets,
                         uint64_t m, uint64_t* out) {
    for (uint64_t k = 0; k < m; k++)
        out[k] = or_count_brute(codes, n, pats + offsets[k], offsets[k + 1] - offsets[k]);
    return OR_OK;
}

/*
 * Work of the count-only backward search with a k-character prefix table
 * (App. D): the table gives the interval of the last k pattern characters
 * without any rank query, then one LF step (two rank queries) is taken per
 * remaining character while the interval is non-empty.  A pattern shorter than
 * k starts from the full interval and steps through all its characters.
 * steps[j] = LF steps of pattern j; returns the total.
 */
uint64_t or_fm_steps(const uint8_t* codes, uint64_t n, const uint64_t* sa, const uint8_t* pats,
                     const uint64_t* offsets, uint64_t m, uint64_t k, uint64_t* steps) {
    uint64_t total = 0;
    for (uint64_t j = 0; j < m; j++) {
        const uint8_t* p = pats + offsets[j];
        uint64_t len = offsets[j + 1] - offsets[j];
        /* longest suffix of p (length t) that occurs in T: intervals only shrink as t grows */
        uint64_t longest = 0;
        for (uint64_t t = 1; t <= len; t++) {
            uint64_t lo, hi;
            or_sa_interval(codes, n, sa, p + (len - t), t, &lo, &hi);
            if (hi > lo) longest = t; else break;
        }
        /* steps t = 1..len run while the interval before step t is non-empty */
        uint64_t run = longest + 1 < len ? longest + 1 : len;
        uint64_t s;
        if (len >= k) s = longest >= k ? run - k : 0;
        else s = run;
        if (steps) steps[j] = s;
        total += s;
    }
    return total;
}
