// kernels.cuh -- launchers shared between the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spr {

constexpr int kDecThreads = 128;             // decode: one thread per block
constexpr int kColStride = kDecThreads + 1;  // padded shared-memory column stride
constexpr int kRowStride = 68;               // decode_list_kernel: words per block row (64 + 4 pad)

// grid for a grid-stride loop over n items, at most per_sm CTAs per SM
int grid_for(int64_t n, int threads, int per_sm);

// Decode the blocks ids[i] (or i) into out + (dst ? dst[i] : i) * 64 for
// i < n, n = *n_dev if n_dev else n_host (n_host bounds the grid).  Nothing
// runs when skip is non-null and *skip != 0.  Out-of-range ids set *bad.
// With planes (the volume's per-block plane counts) the entries are grouped
// by parse length before decoding; the output is the same.
int launch_decode_list(const uint8_t *comp, int64_t nblocks, int rate, const uint32_t *ids,
                       const uint32_t *dst, int64_t n_host, const uint32_t *n_dev,
                       const uint32_t *skip, float *out, unsigned int *bad, cudaStream_t s,
                       const uint8_t *planes = nullptr);

}  // namespace spr
