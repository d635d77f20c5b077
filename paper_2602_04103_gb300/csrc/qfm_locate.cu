// Locate over the QuadFm index: the text positions of every occurrence of a
// pattern, the extension of the count-only index that the paper names as
// future work (Sec. 6).  The paper gives no method; its comparison indexes
// sample the suffix array (App. D, "suffix-array sampling factor"), and so
// does this one, by text position:
//   - rows whose suffix starts at a multiple of s are marked in a bit string
//     over the n + 1 BWT rows, held in a BiRank16 index (so one structure
//     answers both "is row r marked" and "how many marked rows precede r");
//   - samples[rank1(marks, r)] = SA[r] / s for every marked row r.
// A row r is located by LF steps r -> LF(r) (each step moves to the suffix
// one position earlier, SA[LF(r)] = SA[r] - 1) until a marked row r' is
// reached after t steps; then SA[r] = s * samples[rank1(marks, r')] + t, with
// t < s.  The $ row is marked (its suffix starts at 0), so LF never meets it.
//
// qfm_locate: the persistent count kernel writes every pattern's interval,
// an exclusive scan of the counts gives each pattern's first slot in the
// output, and one thread per occurrence walks its row; occurrences of a
// pattern come out in suffix-array row order.
#include "qfm_common.cuh"
#include "qr_scan.cuh"
#include "quadfm.h"

namespace qr {
namespace {

constexpr int kLocThreads = 256;

// Bit r of the mark string: SA[r] is a multiple of s.  The loop is uniform
// over each warp (pad and the stride are multiples of 32), and the warp's
// ballot is one 32-bit word of the string (LSB-first, as qr_build reads it).
__global__ void mark_rows(const uint32_t* __restrict__ sa, uint64_t rows, uint32_t s, uint32_t* __restrict__ words) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t pad = (rows + 31) & ~31ull;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < pad; r += stride) {
        const bool on = r < rows && sa[r] % s == 0;
        const unsigned b = __ballot_sync(0xffffffffu, on);
        if ((threadIdx.x & 31) == 0) words[r >> 5] = b;
    }
}

__global__ void fill_samples(const uint32_t* __restrict__ sa, uint64_t rows, uint32_t s, const uint4* __restrict__ mlines,
                             const uint32_t* __restrict__ msupers, uint32_t* __restrict__ samples) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < rows; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = sa[r];
        if (v % s == 0) samples[birank_rank_paper(mlines, msupers, r)] = v / s;
    }
}

struct LocateArgs {
    FmView v;
    const uint4* __restrict__ mlines;
    const uint32_t* __restrict__ msupers;
    const uint32_t* __restrict__ samples;
    uint32_t s;
    const uint64_t* __restrict__ lohi;  // interval of pattern k at lohi[2k], lohi[2k+1]
    const uint64_t* __restrict__ occ;   // exclusive scan of the counts (m + 1 entries)
    uint64_t m;
    uint64_t total;
    uint64_t* __restrict__ pos;
    uint32_t* status;
};

__global__ void __launch_bounds__(kLocThreads) locate_kernel(LocateArgs a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < a.total; e += stride) {
        // the pattern of occurrence e: the largest k < m with occ[k] <= e
        uint64_t lo = 0, hi = a.m - 1;
        while (lo < hi) {
            const uint64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(a.occ + mid) <= e) lo = mid;
            else hi = mid - 1;
        }
        uint64_t row = __ldg(a.lohi + 2 * lo) + (e - __ldg(a.occ + lo));
        uint32_t steps = 0;
        bool ok = row < a.v.nrows;
        // at most s - 1 steps on a valid index; the bound keeps the loop finite
        while (ok && !birank_bit_paper(a.mlines, row)) {
            if (steps >= a.s) {
                ok = false;
                break;
            }
            row = fm_lf_row(a.v, (uint32_t)row);
            ok = row < a.v.nrows;
            ++steps;
        }
        uint64_t p = ~0ull;
        if (ok) p = (uint64_t)__ldg(a.samples + birank_rank_paper(a.mlines, a.msupers, row)) * a.s + steps;
        else atomicOr(a.status, kStatusTimeout);
        a.pos[e] = p;
    }
}

unsigned grid_for(uint64_t work) {
    uint64_t g = (work + kLocThreads - 1) / kLocThreads;
    const uint64_t cap = (uint64_t)device_props().sms * 16;
    if (g > cap) g = cap;
    return (unsigned)(g ? g : 1);
}

}  // namespace

int build_locate(qfm_index* idx, uint32_t sa_sample, cudaStream_t s) {
    if (!idx->sa) return fail(QR_EINVAL, "locate: the suffix array is gone");
    const uint64_t rows = idx->n + 1;
    const uint64_t nw = (rows + 63) / 64;
    uint64_t* words = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&words, nw * 8, s));
    cudaError_t e = cudaMemsetAsync(words, 0, nw * 8, s);
    if (e == cudaSuccess) {
        mark_rows<<<grid_for(rows), kLocThreads, 0, s>>>(idx->sa, rows, sa_sample, (uint32_t*)words);
        e = cudaGetLastError();
    }
    int rc = e == cudaSuccess ? qr_build_ex(words, rows, 2, 1, QR_LAYOUT_PAPER, s, &idx->marks)
                              : cuda_fail(e, "locate: marks");
    cudaFreeAsync(words, s);
    if (rc != QR_OK) return rc;
    idx->sa_sample = sa_sample;
    idx->nsamples = idx->n / sa_sample + 1;  // positions 0, s, 2s, ... <= n
    QR_CUDA_TRY(cudaMalloc((void**)&idx->samples, idx->nsamples * 4));
    fill_samples<<<grid_for(rows), kLocThreads, 0, s>>>(idx->sa, rows, sa_sample, idx->marks->lines,
                                                        (const uint32_t*)idx->marks->supers, idx->samples);
    QR_CUDA_TRY(cudaGetLastError());
    QR_CUDA_TRY(cudaStreamSynchronize(s));
    return QR_OK;
}

}  // namespace qr

using namespace qr;

extern "C" int qfm_locate(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* occ,
                          uint64_t* positions, uint64_t capacity, uint64_t* total, void* stream) {
    if (!idx || !total) return fail(QR_EINVAL, "qfm_locate: NULL index or total");
    if (!idx->samples) return fail(QR_EINVAL, "qfm_locate: index built without a sampling factor");
    if (!occ || (m > 0 && (!patterns || !offsets))) return fail(QR_EINVAL, "qfm_locate: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    *total = 0;
    if (m == 0) {
        QR_CUDA_TRY(cudaMemsetAsync(occ, 0, 8, s));
        QR_CUDA_TRY(cudaStreamSynchronize(s));
        return QR_OK;
    }
    unsigned long long* queue = nullptr;
    uint64_t* lohi = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&queue, 16, s));
    cudaError_t e = cudaMallocAsync((void**)&lohi, 16 * m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(occ + m, 0, 8, s);
    int rc = QR_OK;
    if (e == cudaSuccess) rc = launch_count(idx, patterns, offsets, m, occ, queue, s, 1, lohi);
    if (e == cudaSuccess && rc == QR_OK) rc = exclusive_scan_u64(occ, occ, m + 1, s);
    uint64_t t = 0;
    if (e == cudaSuccess && rc == QR_OK) e = cudaMemcpyAsync(&t, occ + m, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && rc == QR_OK) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && rc == QR_OK) {
        *total = t;
        if (positions && t > capacity) {
            rc = fail(QR_ERANGE, "qfm_locate: " + std::to_string(t) + " occurrences exceed the capacity of " +
                                     std::to_string(capacity));
        } else if (positions && t > 0) {
            LocateArgs a;
            fm_view(idx, &a.v);
            a.mlines = idx->marks->lines;
            a.msupers = (const uint32_t*)idx->marks->supers;
            a.samples = idx->samples;
            a.s = idx->sa_sample;
            a.lohi = lohi;
            a.occ = occ;
            a.m = m;
            a.total = t;
            a.pos = positions;
            a.status = idx->status;
            locate_kernel<<<grid_for(t), kLocThreads, 0, s>>>(a);
            e = cudaGetLastError();
        }
    }
    if (lohi) cudaFreeAsync(lohi, s);
    cudaFreeAsync(queue, s);
    if (e != cudaSuccess) return cuda_fail(e, "qfm_locate");
    return rc;
}
