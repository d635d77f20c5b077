// Builder of the count-only FM-index (paper App. D): suffix array of T$ by
// prefix doubling on the GPU, BWT with the sentinel's row recorded and its
// symbol stored as code 0, a QuadRank16 index over the BWT, the C array, and
// the 8-mer prefix table.  The paper does not describe suffix sorting; prefix
// doubling (Manber & Myers 1993, in the radix-sort formulation of Larsson &
// Sadakane) maps to GPU sorts: each round sorts (rank[i], rank[i + h]) pairs
// and re-ranks groups of equal keys, doubling the sorted prefix length h.
#include <cub/device/device_radix_sort.cuh>

#include "qfm_common.cuh"
#include "qr_scan.cuh"
#include "quadfm.h"

namespace qr {
namespace {

constexpr int kThreads = 256;
constexpr int kInitChars = 21;  // 21 chars x 3 bits = 63-bit first keys

unsigned blocks_for(uint64_t n) {
    uint64_t b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b > 0x7fffffffull ? 0x7fffffffull : (b ? b : 1));
}

__global__ void check_codes(const uint8_t* __restrict__ t, uint64_t n, uint32_t* __restrict__ bad) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (t[i] > 3) atomicOr(bad, 1u);
}

// key[i] = the first 21 chars of suffix i of T$, 3 bits each ($ and beyond = 0,
// symbol c = c + 1), most significant first; val[i] = i.
__global__ void init_keys(const uint8_t* __restrict__ t, uint64_t n, uint64_t* __restrict__ key,
                          uint32_t* __restrict__ val) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
#pragma unroll
        for (int d = 0; d < kInitChars; d++) {
            const uint64_t p = i + d;
            k = (k << 3) | (p < n ? (uint64_t)t[p] + 1 : 0);
        }
        key[i] = k;
        val[i] = (uint32_t)i;
    }
}

// head[k] = 1 where sorted key k starts a new group of equal keys.
__global__ void mark_heads(const uint64_t* __restrict__ key, uint64_t rows, uint64_t* __restrict__ head) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < rows; k += (uint64_t)gridDim.x * blockDim.x)
        head[k] = (k == 0 || key[k] != key[k - 1]) ? 1 : 0;
}

// rank[sa[k]] = ordinal of the group of row k (inclusive count of heads - 1).
__global__ void scatter_ranks(const uint32_t* __restrict__ sa, const uint64_t* __restrict__ ex,
                              const uint64_t* __restrict__ key, uint64_t rows, uint32_t* __restrict__ rank) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < rows; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t head = (k == 0 || key[k] != key[k - 1]) ? 1 : 0;
        rank[sa[k]] = (uint32_t)(ex[k] + head - 1);
    }
}

__global__ void group_count(const uint64_t* __restrict__ ex, const uint64_t* __restrict__ key, uint64_t rows,
                            uint64_t* __restrict__ groups) {
    const uint64_t k = rows - 1;
    *groups = ex[k] + ((k == 0 || key[k] != key[k - 1]) ? 1 : 0);
}

// Doubling keys: (rank[i], rank[i + h]) packed into 2b bits.  A suffix with
// i + h > n already holds $ among its first h chars, so its group is a
// singleton and its second component is never compared.
__global__ void pair_keys(const uint32_t* __restrict__ rank, uint64_t n, uint64_t h, int b,
                          uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t second = i + h <= n ? rank[i + h] : 0;
        key[i] = ((uint64_t)rank[i] << b) | second;
        val[i] = (uint32_t)i;
    }
}

// BWT of T$ packed 2 bits per row (the $ row stores code 0) and the $ row.
__global__ void pack_bwt(const uint8_t* __restrict__ t, uint64_t n, const uint32_t* __restrict__ sa,
                         uint64_t* __restrict__ words, uint64_t* __restrict__ dollar) {
    const uint64_t rows = n + 1, nw = (rows + 31) / 32;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = 0;
        for (int d = 0; d < 32; d++) {
            const uint64_t k = 32 * w + d;
            if (k >= rows) break;
            const uint32_t s = sa[k];
            if (s == 0) *dollar = k;
            else v |= (uint64_t)(t[s - 1] & 3) << (2 * d);
        }
        words[w] = v;
    }
}

__global__ void histogram4(const uint8_t* __restrict__ t, uint64_t n, unsigned long long* __restrict__ cnt) {
    __shared__ unsigned int local[4];
    if (threadIdx.x < 4) local[threadIdx.x] = 0;
    __syncthreads();
    uint32_t c[4] = {0, 0, 0, 0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        c[t[i] & 3]++;
#pragma unroll
    for (int s = 0; s < 4; s++) atomicAdd(&local[s], c[s]);
    __syncthreads();
    if (threadIdx.x < 4) atomicAdd(&cnt[threadIdx.x], (unsigned long long)local[threadIdx.x]);
}

// Compare the first 8 chars of suffix s of T$ with the 8-mer w (2 bits per
// char, first char most significant): -1 / 0 / +1; a suffix that reaches $
// first sorts before w.
__device__ __forceinline__ int cmp_kmer(const uint8_t* __restrict__ t, uint64_t n, uint64_t s, uint32_t w) {
#pragma unroll
    for (int d = 0; d < kQfmK; d++) {
        if (s + d >= n) return -1;
        const uint32_t a = t[s + d], b = (w >> (2 * (kQfmK - 1 - d))) & 3;
        if (a != b) return a < b ? -1 : 1;
    }
    return 0;
}

// table[w] = [lo, hi): rows of the suffix array whose suffixes start with w.
__global__ void kmer_table(const uint8_t* __restrict__ t, uint64_t n, const uint32_t* __restrict__ sa,
                           uint64_t* __restrict__ table) {
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= kQfmTable) return;
    uint64_t a = 0, b = n + 1;
    while (a < b) {
        const uint64_t mid = a + (b - a) / 2;
        if (cmp_kmer(t, n, sa[mid], w) < 0) a = mid + 1; else b = mid;
    }
    const uint64_t lo = a;
    b = n + 1;
    while (a < b) {
        const uint64_t mid = a + (b - a) / 2;
        if (cmp_kmer(t, n, sa[mid], w) <= 0) a = mid + 1; else b = mid;
    }
    table[2 * w] = lo;
    table[2 * w + 1] = a;
}

int bit_width(uint64_t x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b ? b : 1;
}

struct Scratch {
    cudaStream_t s;
    void* p[8] = {};
    int k = 0;
    cudaError_t alloc(void** out, size_t bytes) {
        cudaError_t e = cudaMallocAsync(out, bytes ? bytes : 16, s);
        if (e == cudaSuccess) p[k++] = *out;
        return e;
    }
    ~Scratch() {
        for (int i = 0; i < k; i++) cudaFreeAsync(p[i], s);
    }
};

}  // namespace

// Suffix array of T$ (rows = n + 1) into sa_out (device, rows uint32).
int build_suffix_array(const uint8_t* d_t, uint64_t n, uint32_t* sa_out, cudaStream_t s) {
    const uint64_t rows = n + 1;
    Scratch sc{s};
    uint64_t *k0, *k1, *groups;
    uint32_t *v1, *rank;
    QR_CUDA_TRY(sc.alloc((void**)&k0, rows * 8));
    QR_CUDA_TRY(sc.alloc((void**)&k1, rows * 8));
    QR_CUDA_TRY(sc.alloc((void**)&v1, rows * 4));
    QR_CUDA_TRY(sc.alloc((void**)&rank, rows * 4));
    QR_CUDA_TRY(sc.alloc((void**)&groups, 8));
    cub::DoubleBuffer<uint64_t> keys(k0, k1);
    cub::DoubleBuffer<uint32_t> vals(sa_out, v1);
    size_t temp_bytes = 0;
    QR_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, keys, vals, rows, 0, 64, s));
    void* temp = nullptr;
    QR_CUDA_TRY(sc.alloc(&temp, temp_bytes));
    const unsigned g = blocks_for(rows);
    init_keys<<<g, kThreads, 0, s>>>(d_t, n, keys.Current(), vals.Current());
    int end_bit = 3 * kInitChars;
    const int b = bit_width(n);  // ranks are group ordinals in [0, n]
    for (uint64_t h = kInitChars;; h *= 2) {
        QR_CUDA_TRY(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, keys, vals, rows, 0, end_bit, s));
        uint64_t* ex = keys.Alternate();  // free after the sort: head flags, then their scan
        mark_heads<<<g, kThreads, 0, s>>>(keys.Current(), rows, ex);
        int rc = exclusive_scan_u64(ex, ex, rows, s);
        if (rc != QR_OK) return rc;
        scatter_ranks<<<g, kThreads, 0, s>>>(vals.Current(), ex, keys.Current(), rows, rank);
        group_count<<<1, 1, 0, s>>>(ex, keys.Current(), rows, groups);
        QR_CUDA_TRY(cudaGetLastError());
        uint64_t ng = 0;
        QR_CUDA_TRY(cudaMemcpyAsync(&ng, groups, 8, cudaMemcpyDeviceToHost, s));
        QR_CUDA_TRY(cudaStreamSynchronize(s));
        if (ng == rows) break;  // every suffix has its own rank: sorted
        if (h >= rows) return fail(QR_ECUDA, "suffix sort did not converge");
        pair_keys<<<g, kThreads, 0, s>>>(rank, n, h, b, keys.Current(), vals.Current());
        end_bit = 2 * b;
    }
    if (vals.Current() != sa_out)
        QR_CUDA_TRY(cudaMemcpyAsync(sa_out, vals.Current(), rows * 4, cudaMemcpyDeviceToDevice, s));
    QR_CUDA_TRY(cudaGetLastError());
    return QR_OK;
}

int build_fm(qfm_index* idx, const uint8_t* d_t, uint64_t n, cudaStream_t s) {
    const uint64_t rows = n + 1;
    Scratch sc{s};
    uint32_t* sa = nullptr;
    uint32_t* bad = nullptr;
    QR_CUDA_TRY(sc.alloc((void**)&bad, 4));
    QR_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, s));
    check_codes<<<blocks_for(n < 4096 * kThreads ? n : 4096 * kThreads), kThreads, 0, s>>>(d_t, n, bad);
    uint32_t hbad = 0;
    QR_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
    QR_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return fail(QR_EINVAL, "qfm_build: text byte > 3");
    QR_CUDA_TRY(cudaMalloc((void**)&sa, rows * 4));
    int rc = build_suffix_array(d_t, n, sa, s);
    if (rc != QR_OK) {
        cudaFree(sa);
        return rc;
    }
    // BWT -> QuadRank16
    uint64_t *words, *dollar;
    unsigned long long* cnt;
    const uint64_t nw = (rows + 31) / 32;
    cudaError_t e = sc.alloc((void**)&words, nw * 8);
    if (e == cudaSuccess) e = sc.alloc((void**)&dollar, 8);
    if (e == cudaSuccess) e = sc.alloc((void**)&cnt, 32);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 32, s);
    if (e != cudaSuccess) {
        cudaFree(sa);
        return cuda_fail(e, "qfm_build: scratch");
    }
    pack_bwt<<<blocks_for(nw), kThreads, 0, s>>>(d_t, n, sa, words, dollar);
    histogram4<<<blocks_for(n < 1024 * kThreads ? n : 1024 * kThreads), kThreads, 0, s>>>(d_t, n, cnt);
    e = cudaMalloc((void**)&idx->table, kQfmTable * 16);
    if (e != cudaSuccess) {
        cudaFree(sa);
        return cuda_fail(e, "qfm_build: table");
    }
    kmer_table<<<(unsigned)(kQfmTable / kThreads), kThreads, 0, s>>>(d_t, n, sa, idx->table);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(sa);
        return cuda_fail(e, "qfm_build: kernels");
    }
    uint64_t hc[4];
    e = cudaMemcpyAsync(hc, cnt, 32, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&idx->dollar_row, dollar, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(sa);
        return cuda_fail(e, "qfm_build: readback");
    }
    idx->C[0] = 1;  // the $ suffix sorts first
    for (int c = 0; c < 4; c++) idx->C[c + 1] = idx->C[c] + hc[c];
    rc = qr_build(words, rows, 4, 1, s, &idx->rank);
    if (rc != QR_OK) {
        cudaFree(sa);
        return rc;
    }
    idx->sa = sa;  // released by the caller unless it keeps it
    return QR_OK;
}

int fm_view(const qfm_index* idx, FmView* v) {
    v->lines = idx->rank->lines;
    v->supers = (const uint4*)idx->rank->supers;
    v->table = idx->table;
    v->nrows = idx->n + 1;
    v->dollar = idx->dollar_row;
    for (int c = 0; c < 4; c++) v->C[c] = idx->C[c];
    return QR_OK;
}

}  // namespace qr
