// mlp.cuh -- the speculation policy MLP on the 5th-generation tensor cores.
//
// The policy is a 12 -> 64 -> 64 -> 2 perceptron with ReLU hidden layers,
// bf16 weights and activations and fp32 accumulation.  A CTA of 128 threads
// evaluates it for a tile of 128 rows (rays): thread t owns row t.  Each layer
// is D[128 x N] = A[128 x K] * B[N x K]^T issued as tcgen05.mma (kind::f16,
// M = 128, K = 16 per instruction) by one thread, A and B in shared memory,
// D in tensor memory; the epilogue reads D back with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31, i.e. rows 32w.., one row per thread), adds the
// bias, applies ReLU, rounds to bf16 and writes the next layer's A.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices (8 bf16 along K), core matrix (r/8, k/8) at
// byte (r/8) * SBO + (k/8) * LBO, row r%8 at 16 * (r%8) within it.  Here
// LBO = 128 (core matrices adjacent along K are contiguous) and SBO = K * 16
// (one 8-row group holds K/8 core matrices).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace spr {
namespace mlp {

constexpr int kIn = 12;       // features
constexpr int kInPad = 16;    // layer 1 K (one MMA)
constexpr int kHid = 64;      // hidden width
constexpr int kOut = 2;       // outputs: log2 k, upper quantile of log2 k
constexpr int kOutPad = 16;   // layer 3 N (the smallest N for M = 128)
constexpr int kRows = 128;    // rows per tile (M)
constexpr int kTmemCols = 64; // fp32 accumulator columns (one layer at a time)

// parameter vector (fp32), PyTorch Linear layout [out][in]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kParams = kOffB3 + kOut;   // 5122

// byte offset of element (r, k) of a K-major operand with K columns
__host__ __device__ constexpr uint32_t kmaj_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory image of the bf16 weights and the fp32 biases
struct Smem {
    alignas(128) uint8_t x[kRows * kInPad * 2];     // A of layer 1
    alignas(128) uint8_t h[kRows * kHid * 2];       // A of layers 2 and 3
    alignas(128) uint8_t w1[kHid * kInPad * 2];     // B of layer 1 (N = 64, K = 16)
    alignas(128) uint8_t w2[kHid * kHid * 2];       // B of layer 2 (N = 64, K = 64)
    alignas(128) uint8_t w3[kOutPad * kHid * 2];    // B of layer 3 (N = 16, K = 64)
    float b1[kHid], b2[kHid], b3[kOutPad];
    alignas(8) unsigned long long mbar;
    uint32_t tmem_base;
    uint32_t error;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, LBO, SBO (bytes, >> 4), the
// version field (1) of the tcgen05 descriptor format, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 D, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for the mbarrier phase with parity `parity`; false when the
// limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Load the parameters into the shared-memory image (all threads).
__device__ inline void load_weights(Smem &S, const float *__restrict__ p)
{
    for (int i = threadIdx.x; i < kHid * kInPad; i += blockDim.x) {
        const int n = i / kInPad, k = i % kInPad;
        const float w = k < kIn ? p[kOffW1 + n * kIn + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(S.w1 + kmaj_off(n, k, kInPad)) = __float2bfloat16_rn(w);
    }
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
        const int n = i / kHid, k = i % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(S.w2 + kmaj_off(n, k, kHid)) = __float2bfloat16_rn(p[kOffW2 + i]);
    }
    for (int i = threadIdx.x; i < kOutPad * kHid; i += blockDim.x) {
        const int n = i / kHid, k = i % kHid;
        const float w = n < kOut ? p[kOffW3 + n * kHid + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(S.w3 + kmaj_off(n, k, kHid)) = __float2bfloat16_rn(w);
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        S.b1[i] = p[kOffB1 + i];
        S.b2[i] = p[kOffB2 + i];
    }
    for (int i = threadIdx.x; i < kOutPad; i += blockDim.x) S.b3[i] = i < kOut ? p[kOffB3 + i] : 0.f;
}

// CTA set-up: mbarrier, TMEM columns (warp 0), weights.  Call with all 128
// threads; ends with a barrier.
__device__ inline void tile_setup(Smem &S, const float *__restrict__ params)
{
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        S.error = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_weights(S, params);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

__device__ inline void tile_teardown(Smem &S)
{
    fence_before();
    __syncthreads();
    fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols)
                     : "memory");
}

// Write this thread's row of the layer-1 input (12 features, rounded to
// bf16, zero padded to 16).
__device__ __forceinline__ void store_features(Smem &S, const float f[kIn])
{
    const int r = threadIdx.x;
    uint4 lo, hi;
    lo.x = pack_bf16x2(f[0], f[1]);
    lo.y = pack_bf16x2(f[2], f[3]);
    lo.z = pack_bf16x2(f[4], f[5]);
    lo.w = pack_bf16x2(f[6], f[7]);
    hi.x = pack_bf16x2(f[8], f[9]);
    hi.y = pack_bf16x2(f[10], f[11]);
    hi.z = 0u;
    hi.w = 0u;
    *reinterpret_cast<uint4 *>(S.x + kmaj_off(r, 0, kInPad)) = lo;
    *reinterpret_cast<uint4 *>(S.x + kmaj_off(r, 8, kInPad)) = hi;
}

// One layer: issue the MMAs (thread 0), wait, and leave D in TMEM.  The
// caller has written A (generic stores) before; this fences them for the
// tensor core.  Returns false when the bounded wait gave up.
__device__ inline bool run_layer(Smem &S, const uint8_t *a, int K, const uint8_t *b, int N, uint32_t &phase)
{
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        const uint32_t id = idesc_bf16(kRows, N);
        const uint32_t sbo = (uint32_t)K * 16u;
        for (int kc = 0; kc < K / 16; ++kc) {
            const uint64_t ad = sdesc(smem_u32(a) + (uint32_t)kc * 256u, 128u, sbo);
            const uint64_t bd = sdesc(smem_u32(b) + (uint32_t)kc * 256u, 128u, sbo);
            mma_bf16(S.tmem_base, ad, bd, id, kc > 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(&S.mbar));
    }
    const bool ok = mbar_wait(smem_u32(&S.mbar), phase, 1u << 24);
    phase ^= 1u;
    fence_after();
    return ok;
}

// Epilogue of a hidden layer: this thread's row of D + bias, ReLU, bf16,
// written as row r of the next layer's A (K = 64).
__device__ inline void hidden_epilogue(Smem &S, const float *bias)
{
    const int r = threadIdx.x;
    const uint32_t lane_base = (uint32_t)((threadIdx.x >> 5) * 32) << 16;
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
        float v[16];
        tmem_ld16(S.tmem_base + lane_base + (uint32_t)c, v);
#pragma unroll
        for (int q = 0; q < 16; q += 8) {
            uint4 o;
            o.x = pack_bf16x2(fmaxf(v[q + 0] + bias[c + q + 0], 0.f), fmaxf(v[q + 1] + bias[c + q + 1], 0.f));
            o.y = pack_bf16x2(fmaxf(v[q + 2] + bias[c + q + 2], 0.f), fmaxf(v[q + 3] + bias[c + q + 3], 0.f));
            o.z = pack_bf16x2(fmaxf(v[q + 4] + bias[c + q + 4], 0.f), fmaxf(v[q + 5] + bias[c + q + 5], 0.f));
            o.w = pack_bf16x2(fmaxf(v[q + 6] + bias[c + q + 6], 0.f), fmaxf(v[q + 7] + bias[c + q + 7], 0.f));
            *reinterpret_cast<uint4 *>(S.h + kmaj_off(r, c + q, kHid)) = o;
        }
    }
}

// The whole network for the tile whose features were stored; this thread's
// two outputs in y.  Returns false (and sets S.error) when a wait gave up;
// the CTA must then stop issuing MMAs.
__device__ inline bool forward_tile(Smem &S, uint32_t &phase, float y[kOut])
{
    if (!run_layer(S, S.x, kInPad, S.w1, kHid, phase)) {
        S.error = 1u;
        return false;
    }
    hidden_epilogue(S, S.b1);
    fence_before();
    if (!run_layer(S, S.h, kHid, S.w2, kHid, phase)) {
        S.error = 1u;
        return false;
    }
    // layer 2's MMAs have completed, so its A (S.h) may be overwritten
    hidden_epilogue(S, S.b2);
    fence_before();
    if (!run_layer(S, S.h, kHid, S.w3, kOutPad, phase)) {
        S.error = 1u;
        return false;
    }
    float v[16];
    tmem_ld16(S.tmem_base + ((uint32_t)((threadIdx.x >> 5) * 32) << 16), v);
    y[0] = v[0] + S.b3[0];
    y[1] = v[1] + S.b3[1];
    fence_before();
    return true;
}

}  // namespace mlp
}  // namespace spr
