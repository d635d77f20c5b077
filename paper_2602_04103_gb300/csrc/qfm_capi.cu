// C-ABI entry points of the QuadFm index (quadfm.h).
#include "qfm_common.cuh"
#include "quadfm.h"

namespace qr {
int build_fm(qfm_index* idx, const uint8_t* d_t, uint64_t n, cudaStream_t s);
int build_locate(qfm_index* idx, uint32_t sa_sample, cudaStream_t s);
int launch_count_stepwise(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                          cudaStream_t s);

namespace {
// Row k of the BWT back from the QuadRank16 lines (slot = k mod 224 + 32).
__global__ void decode_bwt(const uint4* __restrict__ lines, uint64_t rows, uint8_t* __restrict__ out) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < rows; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = div224(k);
        const uint32_t slot = (uint32_t)(k - j * kB4) + 32;
        const uint32_t h = slot >> 7, g = (slot >> 6) & 1, b = slot & 63;
        const uint64_t* w = (const uint64_t*)(lines + 4 * j);
        const uint64_t lo = (~w[4 * h + 2 * g] >> b) & 1, hi = (~w[4 * h + 2 * g + 1] >> b) & 1;
        out[k] = (uint8_t)(lo | (hi << 1));
    }
}

void free_fm(qfm_index* idx) {
    if (!idx) return;
    if (idx->rank) qr_free(idx->rank);
    if (idx->table) cudaFree(idx->table);
    if (idx->sa) cudaFree(idx->sa);
    if (idx->status) cudaFree(idx->status);
    if (idx->marks) qr_free(idx->marks);
    if (idx->samples) cudaFree(idx->samples);
    delete idx;
}
}  // namespace
}  // namespace qr

using namespace qr;

extern "C" {

int qfm_build(const uint8_t* codes, uint64_t n, int codes_on_device, int flags, void* stream, qfm_index** out) {
    return qfm_build_ex(codes, n, codes_on_device, flags, 0, stream, out);
}

int qfm_build_ex(const uint8_t* codes, uint64_t n, int codes_on_device, int flags, uint32_t sa_sample, void* stream,
                 qfm_index** out) {
    if (!out) return fail(QR_EINVAL, "qfm_build: out is NULL");
    *out = nullptr;
    if (n == 0 || n >= 0xFFFFFFFFull - 1) return fail(QR_EINVAL, "qfm_build: need 1 <= n < 2^32 - 1");
    if (!codes) return fail(QR_EINVAL, "qfm_build: codes is NULL");
    if (flags & ~QFM_KEEP_SA) return fail(QR_EINVAL, "qfm_build: unknown flag");
    cudaStream_t s = (cudaStream_t)stream;
    qfm_index* idx = new qfm_index();
    cudaGetDevice(&idx->device);
    idx->n = n;
    cudaError_t e = cudaMalloc((void**)&idx->status, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(idx->status, 0, 64, s);
    const uint8_t* d_t = codes;
    uint8_t* tmp = nullptr;
    if (e == cudaSuccess && !codes_on_device) {
        e = cudaMallocAsync((void**)&tmp, n, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, codes, n, cudaMemcpyHostToDevice, s);
        d_t = tmp;
    }
    if (e != cudaSuccess) {
        if (tmp) cudaFreeAsync(tmp, s);
        cudaStreamSynchronize(s);
        free_fm(idx);
        return cuda_fail(e, "qfm_build: allocation");
    }
    int rc = build_fm(idx, d_t, n, s);
    if (rc == QR_OK && sa_sample > 0) rc = build_locate(idx, sa_sample, s);
    if (tmp) cudaFreeAsync(tmp, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (rc == QR_OK && se != cudaSuccess) rc = cuda_fail(se, "qfm_build: synchronize");
    if (rc != QR_OK) {
        free_fm(idx);
        return rc;
    }
    if (!(flags & QFM_KEEP_SA)) {
        cudaFree(idx->sa);
        idx->sa = nullptr;
    }
    *out = idx;
    return QR_OK;
}

static int check_count(qfm_index* idx, const uint8_t* pat, const uint64_t* off, uint64_t m, uint64_t* out,
                       const char* who) {
    if (!idx) return fail(QR_EINVAL, std::string(who) + ": index is NULL");
    if (m > 0 && (!pat || !off || !out)) return fail(QR_EINVAL, std::string(who) + ": NULL buffer");
    return QR_OK;
}

int qfm_count_ex(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* out,
                 int flags, void* stream) {
    int rc = check_count(idx, patterns, offsets, m, out, "qfm_count");
    if (rc || m == 0) return rc;
    if (flags & ~QFM_BOTH_STRANDS) return fail(QR_EINVAL, "qfm_count_ex: unknown flag");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* queue = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&queue, 16, s));
    cudaError_t e = cudaMemsetAsync(queue, 0, 16, s);
    if (e == cudaSuccess)
        rc = launch_count(idx, patterns, offsets, m, out, queue, s, (flags & QFM_BOTH_STRANDS) ? 2 : 1);
    cudaFreeAsync(queue, s);
    if (e != cudaSuccess) return cuda_fail(e, "qfm_count: queue reset");
    return rc;
}

int qfm_count(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m, uint64_t* out,
              void* stream) {
    return qfm_count_ex(idx, patterns, offsets, m, out, 0, stream);
}

int qfm_count_stepwise(qfm_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t m,
                       uint64_t* out, void* stream) {
    int rc = check_count(idx, patterns, offsets, m, out, "qfm_count_stepwise");
    if (rc || m == 0) return rc;
    return launch_count_stepwise(idx, patterns, offsets, m, out, (cudaStream_t)stream);
}

int qfm_info(const qfm_index* idx, qfm_info_t* info) {
    if (!idx || !info) return fail(QR_EINVAL, "qfm_info: NULL argument");
    info->n = idx->n;
    info->dollar_row = idx->dollar_row;
    for (int c = 0; c < 5; c++) info->C[c] = idx->C[c];
    info->bytes_rank = 64 * idx->rank->nblocks + 16 * idx->rank->nsuper;
    info->bytes_table = kQfmTable * 16;
    info->kmer = kQfmK;
    info->has_sa = idx->sa != nullptr;
    info->sa_sample = (int32_t)idx->sa_sample;
    info->reserved = 0;
    info->bytes_locate = idx->marks ? 64 * idx->marks->nblocks + 4 * idx->marks->nsuper + 4 * idx->nsamples : 0;
    return QR_OK;
}

int qfm_export(const qfm_index* idx, uint32_t* sa, uint8_t* bwt, uint64_t* table, void* stream) {
    if (!idx) return fail(QR_EINVAL, "qfm_export: NULL index");
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t rows = idx->n + 1;
    if (sa) {
        if (!idx->sa) return fail(QR_EINVAL, "qfm_export: the suffix array was not kept (QFM_KEEP_SA)");
        QR_CUDA_TRY(cudaMemcpyAsync(sa, idx->sa, rows * 4, cudaMemcpyDefault, s));
    }
    if (bwt) {
        uint64_t blocks = (rows + 255) / 256;
        if (blocks > 65535) blocks = 65535;
        decode_bwt<<<(unsigned)blocks, 256, 0, s>>>(idx->rank->lines, rows, bwt);
        QR_CUDA_TRY(cudaGetLastError());
    }
    if (table) QR_CUDA_TRY(cudaMemcpyAsync(table, idx->table, kQfmTable * 16, cudaMemcpyDefault, s));
    QR_CUDA_TRY(cudaStreamSynchronize(s));
    return QR_OK;
}

const qr_index* qfm_rank_index(const qfm_index* idx) { return idx ? idx->rank : nullptr; }

int qfm_set_policy(qfm_index* idx, int policy) {
    if (!idx || (policy != kFmPolicyDefault && policy != kFmPolicyKeepIndex && policy != kFmPolicyKeepIndexOnly))
        return fail(QR_EINVAL, "qfm_set_policy: NULL index or unknown policy");
    idx->policy = policy;
    return QR_OK;
}

int qfm_status(qfm_index* idx, void* stream) {
    if (!idx) return fail(QR_EINVAL, "qfm_status: NULL index");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t v = 0;
    QR_CUDA_TRY(cudaMemcpyAsync(&v, idx->status, 4, cudaMemcpyDeviceToHost, s));
    QR_CUDA_TRY(cudaMemsetAsync(idx->status, 0, 4, s));
    QR_CUDA_TRY(cudaStreamSynchronize(s));
    return (int)v;
}

int qfm_free(qfm_index* idx) {
    if (!idx) return QR_OK;
    cudaDeviceSynchronize();
    free_fm(idx);
    return QR_OK;
}

}  // extern "C"
