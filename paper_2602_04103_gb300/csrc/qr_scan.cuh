// Exclusive prefix sum of uint64 arrays on the device (used by the layout
// builders and the FM-index builder).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qr {
// out[i] = in[0] + ... + in[i-1]; in and out may alias.  Temporaries come
// from the stream-ordered pool of s.  Returns QR_OK or an error code.
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s);
}  // namespace qr
