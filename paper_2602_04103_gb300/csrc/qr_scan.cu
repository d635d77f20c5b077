// Three-phase exclusive scan: tiles of 8192 values are scanned by one block
// each (8 serial values per thread + a block-wide warp-shuffle scan), the tile
// totals are scanned recursively, and the tile offsets are added back.
#include "qr_common.cuh"
#include "qr_scan.cuh"

namespace qr {
namespace {

constexpr int kThreads = 1024;
constexpr int kPerThread = 8;
constexpr uint64_t kTile = (uint64_t)kThreads * kPerThread;

__global__ void scan_tiles(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                           uint64_t* __restrict__ tile_sums) {
    __shared__ uint64_t woff[32];
    __shared__ uint64_t tile_total;
    const uint64_t base = blockIdx.x * kTile + (uint64_t)threadIdx.x * kPerThread;
    uint64_t v[kPerThread];
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; k++) {
        uint64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        sum += v[k];
    }
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) woff[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = woff[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        woff[lane] = wi - w;
        if (lane == 31) tile_total = wi;
    }
    __syncthreads();
    uint64_t run = woff[wid] + (incl - sum);
#pragma unroll
    for (int k = 0; k < kPerThread; k++) {
        uint64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = tile_total;
}

__global__ void add_offsets(uint64_t* __restrict__ out, uint64_t n, const uint64_t* __restrict__ offs) {
    const uint64_t base = blockIdx.x * kTile;
    const uint64_t o = offs[blockIdx.x];
    for (uint64_t k = threadIdx.x; k < kTile; k += kThreads) {
        uint64_t i = base + k;
        if (i < n) out[i] += o;
    }
}

}  // namespace

int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s) {
    if (n == 0) return QR_OK;
    const uint64_t tiles = (n + kTile - 1) / kTile;
    if (tiles == 1) {
        scan_tiles<<<1, kThreads, 0, s>>>(in, out, n, nullptr);
        QR_CUDA_TRY(cudaGetLastError());
        return QR_OK;
    }
    uint64_t* sums = nullptr;
    QR_CUDA_TRY(cudaMallocAsync((void**)&sums, sizeof(uint64_t) * tiles, s));
    scan_tiles<<<(unsigned)tiles, kThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    int rc = e == cudaSuccess ? exclusive_scan_u64(sums, sums, tiles, s) : cuda_fail(e, "scan_tiles");
    if (rc == QR_OK) {
        add_offsets<<<(unsigned)tiles, kThreads, 0, s>>>(out, n, sums);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "add_offsets");
    }
    cudaFreeAsync(sums, s);
    return rc;
}

}  // namespace qr
