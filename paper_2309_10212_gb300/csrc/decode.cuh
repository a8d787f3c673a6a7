// decode.cuh -- the renderer's block decoder (Sec. 3.5): the FRC4 blocks of
// a list decoded into 256-byte destination slots, each chunk of the list
// grouped by its blocks' parse lengths.  A template over the functor that
// gives each entry its slot, so that the renderer can hand out its cache
// slots as the decoder reads the misses (csrc/render.cu) and
// spr_volume_decode_blocks can take slots from a list (csrc/codec.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "frc4.cuh"
#include "kernels.cuh"
#include "spr_common.cuh"

namespace spr {

// decode_list_kernel (codec.cu) for lists whose blocks' parse lengths are
// known (the volume's plane counts).  A warp's lanes run the bit-plane loop
// together, so a warp costs about the plane loop of its longest block: lanes
// whose blocks stop after few planes wait for those that parse all 30.  Each
// CTA step therefore takes kSortChunk list entries, counting-sorts them in
// shared memory by their blocks' plane counts, and gives each warp 32
// consecutive entries of that order.  Each entry still goes to its own
// destination slot, slot_of(i, block) (SlotF: begin() once per launch by one
// thread, then slot_of(i, b) once per entry), so the output is the same as
// decode_list_kernel's.  CTAs of 256 threads, one entry per thread and step
// (the rows in dynamic shared memory, 68 KB), so that a list fills the GPU
// with as many threads as decode_list_kernel's.
constexpr int kSortThreads = 256;
constexpr int kSortChunk = kSortThreads;
constexpr size_t kSortRowBytes = sizeof(uint32_t) * kSortThreads * kRowStride;
constexpr uint32_t kNoPlaneKey = 31;   // no entry (plane counts are 0..30)

__device__ __forceinline__ void decode_into_row(const uint8_t *__restrict__ comp, int64_t nblocks, int rate,
                                                int64_t id, const frc4::RegBits &bits, uint32_t *row,
                                                unsigned int *bad)
{
    int emax = 0;
    bool nz = false;
    if (id < nblocks) {   // the parse zeroes the row before it sets bits
        nz = rate <= 2 ? frc4::decode_coeffs(bits, rate, row, 1, &emax)
                       : frc4::decode_block_coeffs(comp + id * 8 * (int64_t)rate, rate, row, 1, &emax);
    } else {
        atomicOr(bad, 1u);
#pragma unroll
        for (int q = 0; q < 16; ++q) reinterpret_cast<uint4 *>(row)[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (nz) {
        float v[64];
        frc4::reconstruct_row(row, emax, v);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            reinterpret_cast<uint4 *>(row)[q] =
                make_uint4(__float_as_uint(v[4 * q]), __float_as_uint(v[4 * q + 1]), __float_as_uint(v[4 * q + 2]),
                           __float_as_uint(v[4 * q + 3]));
    }
}

template <class SlotF>
__global__ void __launch_bounds__(kSortThreads, 3) decode_sorted_kernel(
    const uint8_t *__restrict__ comp, int64_t nblocks, int rate, const uint8_t *__restrict__ planes,
    const uint32_t *__restrict__ ids, SlotF slot_of, int64_t n_host, const uint32_t *n_dev, const uint32_t *skip,
    float *__restrict__ out, unsigned int *bad)
{
    extern __shared__ __align__(16) uint32_t rows_s[];   // kSortThreads rows of kRowStride words
    // the chunk's entries in sorted order: block id, destination slot and
    // (rate <= 2) the bit stream, loaded before the sort by the thread that
    // read the entry, so the parse does not wait on a second round of loads
    __shared__ uint4 s_bits[kSortChunk];
    __shared__ uint32_t s_id[kSortChunk];
    __shared__ uint32_t s_slot[kSortChunk];
    __shared__ uint32_t s_off[32];
    if (skip && *skip) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) slot_of.begin();
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    uint32_t *row = rows_s + threadIdx.x * kRowStride;
    const uint32_t *wrows = rows_s + wid * 32 * kRowStride;
    const int64_t bytes = 8 * (int64_t)rate;
    constexpr int kRounds = kSortChunk / kSortThreads;
    for (int64_t c0 = (int64_t)blockIdx.x * kSortChunk; c0 < n; c0 += (int64_t)gridDim.x * kSortChunk) {
        const int m = n - c0 < kSortChunk ? (int)(n - c0) : kSortChunk;
        if (threadIdx.x < 32) s_off[threadIdx.x] = 0u;
        __syncthreads();   // the previous step's reads of the shared arrays are done
        // each entry: its block, slot, stream and key (the block's plane
        // count); per-key counts
        uint32_t key[kRounds], eid[kRounds], eslot[kRounds];
        uint4 ebits[kRounds];
#pragma unroll
        for (int j = 0; j < kRounds; ++j) {
            const int l = j * kSortThreads + threadIdx.x;
            key[j] = kNoPlaneKey;
            eid[j] = 0u;
            eslot[j] = 0u;
            ebits[j] = make_uint4(0u, 0u, 0u, 0u);
            if (l < m) {
                eid[j] = ids ? ids[c0 + l] : (uint32_t)(c0 + l);
                key[j] = 0u;
                if ((int64_t)eid[j] < nblocks) {
                    key[j] = planes[eid[j]];
                    if (rate == 2)
                        ebits[j] = __ldg(reinterpret_cast<const uint4 *>(comp + (int64_t)eid[j] * bytes));
                    else if (rate == 1) {
                        const uint2 h = __ldg(reinterpret_cast<const uint2 *>(comp + (int64_t)eid[j] * bytes));
                        ebits[j] = make_uint4(h.x, h.y, 0u, 0u);
                    }
                }
                // after the loads above, which then need not wait on the
                // functor's stores
                eslot[j] = slot_of(c0 + l, eid[j]);
            }
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key[j]);
            if (key[j] != kNoPlaneKey && (peers & below) == 0) atomicAdd(&s_off[key[j]], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (wid == 0) {   // exclusive offsets of the keys
            const uint32_t v = s_off[lane];
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            s_off[lane] = incl - v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kRounds; ++j) {
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key[j]);
            const int leader = __ffs(peers) - 1;
            uint32_t at = 0;
            if (key[j] != kNoPlaneKey && lane == leader) at = atomicAdd(&s_off[key[j]], (uint32_t)__popc(peers));
            at = __shfl_sync(0xFFFFFFFFu, at, leader);
            if (key[j] != kNoPlaneKey) {
                const uint32_t pos = at + __popc(peers & below);
                s_bits[pos] = ebits[j];
                s_id[pos] = eid[j];
                s_slot[pos] = eslot[j];
            }
        }
        __syncthreads();
        // warp wid takes sorted positions r * kSortThreads + 32 * wid + lane
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int q0 = r * kSortThreads + wid * 32;
            if (q0 >= m) break;   // the same for the whole warp
            const int q = q0 + lane;
            uint32_t slot = 0u;
            if (q < m) {
                const uint4 b4 = s_bits[q];
                const frc4::RegBits bits{b4.x, b4.y, b4.z, b4.w};
                slot = s_slot[q];
                decode_into_row(comp, nblocks, rate, (int64_t)s_id[q], bits, row, bad);
            }
            __syncwarp();
            // blocks t and t + 1 of the warp per step: lanes 0-15 and 16-31
            // each move one 16-byte quarter-row
            const int cnt = m - q0 < 32 ? m - q0 : 32;
            const int half = lane >> 4, qq = lane & 15;
            for (int t = 0; t < cnt; t += 2) {
                const int blk = t + half;
                const uint32_t sl = __shfl_sync(0xFFFFFFFFu, slot, blk & 31);
                if (blk < cnt) {
                    const uint4 w = reinterpret_cast<const uint4 *>(wrows + blk * kRowStride)[qq];
                    reinterpret_cast<uint4 *>(out + (int64_t)sl * 64)[qq] = w;
                }
            }
            __syncwarp();
        }
    }
}


// The kernel's dynamic shared memory (above the 48 KB default) and its CTAs
// per SM (8 waves of the resident ones), once per instantiation and device
// (a function attribute holds for the device current when it is set).  Call
// it with the device current, outside stream capture, before the first
// launch there; later calls on that device only read the cached value.
constexpr int kSortMaxDevices = 64;

template <class SlotF>
inline int decode_sorted_prepare(int *per_sm)
{
    static int cached[kSortMaxDevices] = {};
    int dev = 0;
    SPR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kSortMaxDevices)
        return set_error(SPR_ERR_INVALID_ARG, "device ordinal %d beyond the %d supported", dev, kSortMaxDevices);
    if (cached[dev] == 0) {
        SPR_CUDA_TRY(cudaFuncSetAttribute(decode_sorted_kernel<SlotF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSortRowBytes));
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decode_sorted_kernel<SlotF>, kSortThreads,
                                                          kSortRowBytes) != cudaSuccess ||
            nb < 1)
            nb = 1;
        cached[dev] = nb * 8;
    }
    if (per_sm) *per_sm = cached[dev];
    return SPR_OK;
}

// Decode list entries i < n (n = *n_dev if n_dev else n_host; n_host bounds
// the grid) of blocks ids[i] (or i) into out + slot_of(i, id) * 64.
template <class SlotF>
inline int launch_decode_sorted(const uint8_t *comp, int64_t nblocks, int rate, const uint8_t *planes,
                                const uint32_t *ids, SlotF slot_of, int64_t n_host, const uint32_t *n_dev,
                                const uint32_t *skip, float *out, unsigned int *bad, cudaStream_t s)
{
    if (n_host <= 0) return SPR_OK;
    int per_sm = 0;
    SPR_TRY(decode_sorted_prepare<SlotF>(&per_sm));
    decode_sorted_kernel<SlotF><<<grid_for(n_host, kSortChunk, per_sm), kSortThreads, kSortRowBytes, s>>>(
        comp, nblocks, rate, planes, ids, slot_of, n_host, n_dev, skip, out, bad);
    SPR_CUDA_TRY(cudaGetLastError());
    return SPR_OK;
}

}  // namespace spr
