// codec.cu -- FRC4 encode/decode kernels and volume creation (Sec. 3.1).
//
// create_volume decodes every block once to get its value range, then builds
// the fine grid (one cell per block) and the coarse grid (one cell per 4^3
// blocks), each cell's range combined with its +x/+y/+z neighbours' ranges.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "decode.cuh"
#include "frc4.cuh"
#include "kernels.cuh"
#include "spr_common.cuh"

namespace spr {

VolGeom make_geom(const int32_t dims[3], int rate)
{
    VolGeom g{};
    g.rate = rate;
    g.nblocks = 1;
    g.ncoarse = 1;
    for (int a = 0; a < 3; ++a) {
        g.dims[a] = dims[a];
        g.nb[a] = (dims[a] + 3) / 4;
        g.nc[a] = (g.nb[a] + 3) / 4;
        g.tb[a] = (dims[a] - 1 + 3) / 4;
        g.tc[a] = (g.tb[a] + 3) / 4;
        g.nblocks *= g.nb[a];
        g.ncoarse *= g.nc[a];
    }
    return g;
}

// ---------------------------------------------------------------- kernels
// raw range of each block: min/max of its decoded in-domain voxels; and the
// number of bit planes its parse reads
__global__ void __launch_bounds__(kDecThreads) range_kernel(const uint8_t *__restrict__ comp,
                                                            VolGeom g, float2 *__restrict__ raw,
                                                            uint8_t *__restrict__ planes)
{
    __shared__ uint32_t col_s[64 * kColStride];
    uint32_t *col = col_s + threadIdx.x;
    const int64_t bytes = 8 * (int64_t)g.rate;
    for (int64_t b = (int64_t)blockIdx.x * kDecThreads + threadIdx.x; b < g.nblocks;
         b += (int64_t)gridDim.x * kDecThreads) {
        int emax = 0, np = 0;
        float mn = 0.0f, mx = 0.0f;
        const bool nz = frc4::decode_block_coeffs(comp + b * bytes, g.rate, col, kColStride, &emax, &np);
        planes[b] = (uint8_t)np;
        if (nz) {
            int64_t bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / ((int64_t)g.nb[0] * g.nb[1]);
            int ex = min(4, (int)(g.dims[0] - 4 * bx));
            int ey = min(4, (int)(g.dims[1] - 4 * by));
            int ez = min(4, (int)(g.dims[2] - 4 * bz));
            float v[64];
            frc4::reconstruct(col, kColStride, emax, v);
            mn = INFINITY;
            mx = -INFINITY;
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                bool in = (i & 3) < ex && ((i >> 2) & 3) < ey && (i >> 4) < ez;
                if (in) {
                    mn = fminf(mn, v[i]);
                    mx = fmaxf(mx, v[i]);
                }
            }
        }
        raw[b] = make_float2(mn, mx);
    }
}

// union of a cell's range with its +x/+y/+z face, edge and corner neighbours
__global__ void plus_union_kernel(const float2 *__restrict__ in, int nx, int ny, int nz,
                                  float2 *__restrict__ out)
{
    int64_t n = (int64_t)nx * ny * nz;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
        float mn = INFINITY, mx = -INFINITY;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            int xx = x + (o & 1), yy = y + ((o >> 1) & 1), zz = z + (o >> 2);
            if (xx < nx && yy < ny && zz < nz) {
                float2 r = in[xx + (int64_t)nx * (yy + (int64_t)ny * zz)];
                mn = fminf(mn, r.x);
                mx = fmaxf(mx, r.y);
            }
        }
        out[c] = make_float2(mn, mx);
    }
}

// range of the 4^3 blocks of each coarse cell
__global__ void coarse_raw_kernel(const float2 *__restrict__ raw, VolGeom g, float2 *__restrict__ craw)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncoarse;
         c += (int64_t)gridDim.x * blockDim.x) {
        int cx = (int)(c % g.nc[0]), cy = (int)((c / g.nc[0]) % g.nc[1]),
            cz = (int)(c / ((int64_t)g.nc[0] * g.nc[1]));
        float mn = INFINITY, mx = -INFINITY;
        for (int z = 4 * cz; z < min(4 * cz + 4, g.nb[2]); ++z)
            for (int y = 4 * cy; y < min(4 * cy + 4, g.nb[1]); ++y)
                for (int x = 4 * cx; x < min(4 * cx + 4, g.nb[0]); ++x) {
                    float2 r = raw[x + (int64_t)g.nb[0] * (y + (int64_t)g.nb[1] * z)];
                    mn = fminf(mn, r.x);
                    mx = fmaxf(mx, r.y);
                }
        craw[c] = make_float2(mn, mx);
    }
}

// encode: one thread per block, edge-replicating partial blocks
template <class T>
__global__ void encode_kernel(const T *__restrict__ vol, VolGeom g, uint8_t *__restrict__ out,
                              unsigned int *bad)
{
    const int64_t bytes = 8 * (int64_t)g.rate;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < g.nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / ((int64_t)g.nb[0] * g.nb[1]);
        float v[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            int64_t x = min(4 * bx + (i & 3), (int64_t)g.dims[0] - 1);
            int64_t y = min(4 * by + ((i >> 2) & 3), (int64_t)g.dims[1] - 1);
            int64_t z = min(4 * bz + (i >> 4), (int64_t)g.dims[2] - 1);
            T raw = vol[x + (int64_t)g.dims[0] * (y + (int64_t)g.dims[1] * z)];
            if constexpr (sizeof(T) == 1)
                v[i] = __fdiv_rn((float)raw, 255.0f);
            else
                v[i] = (float)raw;
        }
        uint32_t *w = reinterpret_cast<uint32_t *>(out + b * bytes);
        if (!frc4::encode_block(v, g.rate, w)) atomicOr(bad, 1u);
    }
}

// decode blocks ids[i] (or i) to out + dst[i]*64 (or i*64), a warp writing
// its 32 blocks with coalesced stores.  Each lane loads its own destination
// slot once and the warp shares them by shuffles.  At rates <= 2 the loads
// are software-pipelined: while a lane decodes item k, the bitstream of item
// k+1 and the block id of item k+2 are in flight.
__device__ __forceinline__ int64_t dec_id(const uint32_t *ids, int64_t i, int64_t n)
{
    return i < n ? (ids ? (int64_t)ids[i] : i) : -1;
}

// One thread decodes one block into its own row of shared memory (64
// coefficient words, padded to 68 so that the 128-bit accesses of a quarter
// warp hit 32 distinct banks); the warp then writes its blocks out two per
// instruction, 16 bytes per lane.  Rates <= 2 keep the whole stream in
// registers (one 128-bit load, software-pipelined one block ahead).  Six
// CTAs per SM (shared memory allows six; the register cap keeps it).
__global__ void __launch_bounds__(kDecThreads, 6) decode_list_kernel(
    const uint8_t *__restrict__ comp, int64_t nblocks, int rate, const uint32_t *__restrict__ ids,
    const uint32_t *__restrict__ dst_ids, int64_t n_host, const uint32_t *n_dev,
    const uint32_t *skip, float *__restrict__ out, unsigned int *bad)
{
    __shared__ __align__(16) uint32_t rows_s[kDecThreads * kRowStride];
    if (skip && *skip) return;
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *row = rows_s + threadIdx.x * kRowStride;
    const uint32_t *wrows = rows_s + wid * 32 * kRowStride;
    const int64_t bytes = 8 * (int64_t)rate;
    const int64_t stride = (int64_t)gridDim.x * kDecThreads;
    const bool reg = rate <= 2;
    int64_t base = (int64_t)blockIdx.x * kDecThreads + wid * 32;
    int64_t id = dec_id(ids, base + lane, n);
    int64_t id_next = dec_id(ids, base + stride + lane, n);
    frc4::RegBits cur{0u, 0u, 0u, 0u};
    if (reg && id >= 0 && id < nblocks) cur = frc4::load_reg_bits(comp + id * bytes, rate);
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (; base < n; base += stride) {
        const int64_t i = base + lane;
        // loads for the next items, consumed one and two iterations later
        frc4::RegBits nxt{0u, 0u, 0u, 0u};
        if (reg && id_next >= 0 && id_next < nblocks) nxt = frc4::load_reg_bits(comp + id_next * bytes, rate);
        const int64_t id_after = dec_id(ids, base + 2 * stride + lane, n);
        const uint32_t my_slot = i < n ? (dst_ids ? dst_ids[i] : (uint32_t)i) : 0u;
        if (i < n) {
            int emax = 0;
            bool nz = false;
            // the parse zeroes the row before it sets bits
            if (id < nblocks) {
                nz = reg ? frc4::decode_coeffs(cur, rate, row, 1, &emax)
                         : frc4::decode_block_coeffs(comp + id * bytes, rate, row, 1, &emax);
            } else {
                atomicOr(bad, 1u);
#pragma unroll
                for (int q = 0; q < 16; ++q) reinterpret_cast<uint4 *>(row)[q] = zero4;
            }
            if (nz) {
                float v[64];
                frc4::reconstruct_row(row, emax, v);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    reinterpret_cast<uint4 *>(row)[q] =
                        make_uint4(__float_as_uint(v[4 * q]), __float_as_uint(v[4 * q + 1]),
                                   __float_as_uint(v[4 * q + 2]), __float_as_uint(v[4 * q + 3]));
            }
        }
        __syncwarp();
        // blocks t and t + 1 of the warp per step: lanes 0-15 and 16-31 each
        // move one 16-byte quarter-row
        const int m = n - base < 32 ? (int)(n - base) : 32;
        const int half = lane >> 4, q = lane & 15;
        for (int t = 0; t < m; t += 2) {
            const int blk = t + half;
            const uint32_t slot = __shfl_sync(0xFFFFFFFFu, my_slot, blk & 31);
            if (blk < m) {
                const uint4 w = reinterpret_cast<const uint4 *>(wrows + blk * kRowStride)[q];
                reinterpret_cast<uint4 *>(out + (int64_t)slot * 64)[q] = w;
            }
        }
        __syncwarp();
        cur = nxt;
        id = id_next;
        id_next = id_after;
    }
}

int grid_for(int64_t n, int threads, int per_sm)
{
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)device_sm_count() * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

static int check_dims_rate(const int32_t dims[3], int rate)
{
    if (!dims) return set_error(SPR_ERR_INVALID_ARG, "dims is NULL");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || dims[a] > 4096)
            return set_error(SPR_ERR_INVALID_ARG, "dims[%d] = %d outside [2, 4096]", a, dims[a]);
    if (rate < 1 || rate > 32) return set_error(SPR_ERR_INVALID_ARG, "rate %d outside [1, 32]", rate);
    return SPR_OK;
}

template <class T>
static int encode_impl(const T *vol, const int32_t dims[3], int rate, uint8_t *out, spr_stream st)
{
    clear_error();
    SPR_TRY(check_dims_rate(dims, rate));
    if (!vol || !out) return set_error(SPR_ERR_INVALID_ARG, "NULL buffer");
    cudaStream_t s = as_stream(st);
    VolGeom g = make_geom(dims, rate);
    DevBuf flag;
    SPR_TRY(buf_alloc(flag, sizeof(unsigned int), s));
    SPR_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(unsigned int), s));
    encode_kernel<T><<<grid_for(g.nblocks, 128, 16), 128, 0, s>>>(vol, g, out, flag.as<unsigned int>());
    SPR_CUDA_TRY(cudaGetLastError());
    unsigned int bad = 0;
    SPR_CUDA_TRY(cudaMemcpyAsync(&bad, flag.p, sizeof bad, cudaMemcpyDeviceToHost, s));
    SPR_CUDA_TRY(cudaStreamSynchronize(s));
    buf_free(flag, s);
    if (bad) return set_error(SPR_ERR_INVALID_ARG, "volume holds non-finite values");
    return SPR_OK;
}

// destination slot of list entry i: dst[i], or i
struct ListSlot {
    const uint32_t *dst;
    __device__ void begin() const {}
    __device__ uint32_t operator()(int64_t i, uint32_t) const { return dst ? dst[i] : (uint32_t)i; }
};

int launch_decode_list(const uint8_t *comp, int64_t nblocks, int rate, const uint32_t *ids,
                       const uint32_t *dst, int64_t n_host, const uint32_t *n_dev,
                       const uint32_t *skip, float *out, unsigned int *bad, cudaStream_t s,
                       const uint8_t *planes)
{
    if (n_host <= 0) return SPR_OK;
    if (planes)
        return launch_decode_sorted(comp, nblocks, rate, planes, ids, ListSlot{dst}, n_host, n_dev, skip, out, bad,
                                    s);
    // kDecWaves waves of the CTAs resident at once (shared memory bound), so
    // that an SM whose CTAs finish early takes new ones: in a render the
    // decode runs beside the grouping branch, whose kernels hold SMs when it
    // starts, and one exact wave then left CTAs with 4 blocks per thread
    // starting late (paper scale 0.959 -> 0.925 ms with 8 waves; the decode
    // of 16.8 M consecutive blocks 2,026 -> 2,205 GB/s)
    constexpr int kDecWaves = 8;
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decode_list_kernel, kDecThreads, 0) != cudaSuccess ||
            nb < 1)
            nb = 1;
        per_sm = nb * kDecWaves;
    }
    decode_list_kernel<<<grid_for(n_host, kDecThreads, per_sm), kDecThreads, 0, s>>>(
        comp, nblocks, rate, ids, dst, n_host, n_dev, skip, out, bad);
    SPR_CUDA_TRY(cudaGetLastError());
    return SPR_OK;
}

}  // namespace spr

using namespace spr;

extern "C" int spr_encode_f32(const float *vol, const int32_t dims[3], int rate, uint8_t *out,
                              spr_stream stream)
{
    return encode_impl<float>(vol, dims, rate, out, stream);
}

extern "C" int spr_encode_u8(const uint8_t *vol, const int32_t dims[3], int rate, uint8_t *out,
                             spr_stream stream)
{
    return encode_impl<uint8_t>(vol, dims, rate, out, stream);
}

extern "C" int spr_decode_blocks(const uint8_t *blocks, int64_t n_blocks, int rate,
                                 const uint32_t *ids, int64_t n, float *out, spr_stream stream)
{
    clear_error();
    if (!blocks || !out || n < 0 || n_blocks < 1)
        return set_error(SPR_ERR_INVALID_ARG, "bad decode arguments");
    if (rate < 1 || rate > 32) return set_error(SPR_ERR_INVALID_ARG, "rate %d outside [1, 32]", rate);
    if (!ids && n > n_blocks) return set_error(SPR_ERR_INVALID_ARG, "n exceeds the block count");
    cudaStream_t s = as_stream(stream);
    DevBuf flag;
    SPR_TRY(buf_alloc(flag, sizeof(unsigned int), s));
    SPR_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(unsigned int), s));
    int rc = launch_decode_list(blocks, n_blocks, rate, ids, nullptr, n, nullptr, nullptr, out,
                                flag.as<unsigned int>(), s);
    unsigned int bad = 0;
    if (rc == SPR_OK) {
        cudaError_t e = cudaMemcpyAsync(&bad, flag.p, sizeof bad, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "decode: %s", cudaGetErrorString(e));
    }
    buf_free(flag, s);
    if (rc == SPR_OK && bad) rc = set_error(SPR_ERR_INVALID_ARG, "a block id is out of range");
    return rc;
}

extern "C" int spr_volume_decode_blocks(const spr_volume *v, const uint32_t *ids, int64_t n, float *out,
                                        spr_stream stream)
{
    clear_error();
    if (!v || n < 0 || (n > 0 && !out)) return set_error(SPR_ERR_INVALID_ARG, "bad decode arguments");
    if (!ids && n > v->g.nblocks) return set_error(SPR_ERR_INVALID_ARG, "n exceeds the block count");
    if (n == 0) return SPR_OK;
    cudaStream_t s = as_stream(stream);
    DevBuf flag;
    SPR_TRY(buf_alloc(flag, sizeof(unsigned int), s));
    int rc = SPR_OK;
    cudaError_t e = cudaMemsetAsync(flag.p, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "decode: %s", cudaGetErrorString(e));
    if (rc == SPR_OK)
        rc = launch_decode_list(v->comp.as<uint8_t>(), v->g.nblocks, v->g.rate, ids, nullptr, n, nullptr, nullptr,
                                out, flag.as<unsigned int>(), s, v->planes.as<uint8_t>());
    unsigned int bad = 0;
    if (rc == SPR_OK) {
        e = cudaMemcpyAsync(&bad, flag.p, sizeof bad, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "decode: %s", cudaGetErrorString(e));
    }
    buf_free(flag, s);
    if (rc == SPR_OK && bad) rc = set_error(SPR_ERR_INVALID_ARG, "a block id is out of range");
    return rc;
}

extern "C" int spr_create_volume(const spr_volume_desc *desc, const void *blocks, size_t nbytes,
                                 int blocks_on_device, spr_stream stream, spr_volume **out)
{
    clear_error();
    if (!desc || !blocks || !out) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    SPR_TRY(check_dims_rate(desc->dims, desc->rate));
    if (desc->codec != SPR_CODEC_FRC4) return set_error(SPR_ERR_INVALID_ARG, "unknown codec %d", desc->codec);
    VolGeom g = make_geom(desc->dims, desc->rate);
    size_t need = (size_t)g.nblocks * 8 * (size_t)g.rate;
    if (nbytes != need)
        return set_error(SPR_ERR_INVALID_ARG, "expected %zu compressed bytes, got %zu", need, nbytes);
    cudaStream_t s = as_stream(stream);
    SPR_TRY(decode_sorted_prepare<ListSlot>(nullptr));
    spr_volume *v = new (std::nothrow) spr_volume();
    if (!v) return set_error(SPR_ERR_OUT_OF_MEMORY, "host allocation failed");
    v->g = g;
    DevBuf raw, craw;
    int rc = SPR_OK;
    auto fail = [&](int code) {
        buf_free(raw, s);
        buf_free(craw, s);
        buf_free(v->comp, s);
        buf_free(v->fine, s);
        buf_free(v->coarse, s);
        buf_free(v->planes, s);
        delete v;
        return code;
    };
    if ((rc = buf_alloc(v->comp, need, s)) || (rc = buf_alloc(v->fine, sizeof(float2) * g.nblocks, s)) ||
        (rc = buf_alloc(v->planes, (size_t)g.nblocks, s)) ||
        (rc = buf_alloc(v->coarse, sizeof(float2) * g.ncoarse, s)) ||
        (rc = buf_alloc(raw, sizeof(float2) * g.nblocks, s)) ||
        (rc = buf_alloc(craw, sizeof(float2) * g.ncoarse, s)))
        return fail(rc);
    cudaError_t e = cudaMemcpyAsync(v->comp.p, blocks, need,
                                    blocks_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(set_error(SPR_ERR_CUDA, "copy of blocks: %s", cudaGetErrorString(e)));
    range_kernel<<<grid_for(g.nblocks, kDecThreads, 8), kDecThreads, 0, s>>>(v->comp.as<uint8_t>(), g,
                                                                           raw.as<float2>(),
                                                                           v->planes.as<uint8_t>());
    plus_union_kernel<<<grid_for(g.nblocks, 256, 8), 256, 0, s>>>(raw.as<float2>(), g.nb[0], g.nb[1], g.nb[2],
                                                                 v->fine.as<float2>());
    coarse_raw_kernel<<<grid_for(g.ncoarse, 256, 8), 256, 0, s>>>(raw.as<float2>(), g, craw.as<float2>());
    plus_union_kernel<<<grid_for(g.ncoarse, 256, 8), 256, 0, s>>>(craw.as<float2>(), g.nc[0], g.nc[1],
                                                                 g.nc[2], v->coarse.as<float2>());
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(set_error(SPR_ERR_CUDA, "volume setup: %s", cudaGetErrorString(e)));
    buf_free(raw, s);
    buf_free(craw, s);
    *out = v;
    return SPR_OK;
}

extern "C" int spr_destroy_volume(spr_volume *v)
{
    clear_error();
    if (!v) return SPR_OK;
    cudaDeviceSynchronize();
    buf_free(v->comp, nullptr);
    buf_free(v->fine, nullptr);
    buf_free(v->coarse, nullptr);
    buf_free(v->planes, nullptr);
    delete v;
    return SPR_OK;
}

extern "C" int spr_volume_ranges(const spr_volume *v, float *fine_host, float *coarse_host,
                                 spr_stream stream)
{
    clear_error();
    if (!v) return set_error(SPR_ERR_INVALID_ARG, "NULL volume");
    cudaStream_t s = as_stream(stream);
    if (fine_host)
        SPR_CUDA_TRY(cudaMemcpyAsync(fine_host, v->fine.p, sizeof(float2) * v->g.nblocks,
                                     cudaMemcpyDeviceToHost, s));
    if (coarse_host)
        SPR_CUDA_TRY(cudaMemcpyAsync(coarse_host, v->coarse.p, sizeof(float2) * v->g.ncoarse,
                                     cudaMemcpyDeviceToHost, s));
    SPR_CUDA_TRY(cudaStreamSynchronize(s));
    return SPR_OK;
}

namespace spr {
// per block: is its fine range holding the isovalue (active), and is it
// active or the +x/+y/+z face, edge or corner neighbour of an active block
// (needed: its values enter an active block's cells)
__global__ void count_active_kernel(const float2 *__restrict__ fine, VolGeom g, float iso,
                                    unsigned long long *counts)
{
    const int64_t nb0 = g.nb[0], nb1 = g.nb[1], nb2 = g.nb[2];
    unsigned long long na = 0, nn = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < g.nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = b % nb0, y = (b / nb0) % nb1, z = b / (nb0 * nb1);
        bool need = false;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int64_t xs = x - (o & 1), ys = y - ((o >> 1) & 1), zs = z - (o >> 2);
            if (xs < 0 || ys < 0 || zs < 0) continue;
            const float2 r = fine[xs + nb0 * (ys + nb1 * zs)];
            const bool act = r.x <= iso && iso <= r.y;
            if (o == 0) na += act;
            need = need || act;
        }
        nn += need;
        (void)nb2;
    }
    for (int off = 16; off; off >>= 1) {
        na += __shfl_down_sync(0xFFFFFFFFu, na, off);
        nn += __shfl_down_sync(0xFFFFFFFFu, nn, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (na) atomicAdd(&counts[0], na);
        if (nn) atomicAdd(&counts[1], nn);
    }
}
}  // namespace spr

extern "C" int spr_count_active_blocks(const spr_volume *v, float iso, int64_t *n_active, int64_t *n_needed,
                                       spr_stream stream)
{
    clear_error();
    if (!v || !std::isfinite(iso)) return set_error(SPR_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = as_stream(stream);
    DevBuf counts;
    SPR_TRY(buf_alloc(counts, 2 * sizeof(unsigned long long), s));
    unsigned long long h[2] = {0, 0};
    int rc = SPR_OK;
    cudaError_t e = cudaMemsetAsync(counts.p, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        count_active_kernel<<<grid_for(v->g.nblocks, 256, 8), 256, 0, s>>>(v->fine.as<float2>(), v->g, iso,
                                                                           counts.as<unsigned long long>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts.p, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "count_active: %s", cudaGetErrorString(e));
    buf_free(counts, s);
    if (rc == SPR_OK) {
        if (n_active) *n_active = (int64_t)h[0];
        if (n_needed) *n_needed = (int64_t)h[1];
    }
    return rc;
}

extern "C" int spr_volume_shape(const spr_volume *v, int64_t nb[3], int64_t nc[3])
{
    clear_error();
    if (!v) return set_error(SPR_ERR_INVALID_ARG, "NULL volume");
    for (int a = 0; a < 3; ++a) {
        if (nb) nb[a] = v->g.nb[a];
        if (nc) nc[a] = v->g.nc[a];
    }
    return SPR_OK;
}
