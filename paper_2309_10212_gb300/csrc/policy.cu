// policy.cu -- the speculation policy's standalone inference and training.
//
// The paper leaves a per-ray speculation count to future work (Sec. 6); the
// renderer's learned mode (SPR_SPEC_LEARNED) predicts it with the MLP of
// mlp.cuh.  This file has the MLP on caller features (the same tensor-core
// tile as the renderer's policy kernel) and its training: a fused forward and
// backward pass in fp32 on the CUDA cores, gradients summed per CTA, and an
// Adam update, all in hand-written kernels.
//
// Loss per sample with target t = log2(min(label, 64)) (label = the visible
// blocks the ray still needed): (y0 - t)^2 for the first output and the
// pinball loss of quantile tau, max(tau (t - y1), (tau - 1)(t - y1)), for the
// second; both averaged over the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.cuh"
#include "spr_common.cuh"

using namespace spr;

namespace {

using namespace spr::mlp;

__global__ void __launch_bounds__(128) forward_kernel(const float *__restrict__ params, const float *__restrict__ x,
                                                      int64_t n, float *__restrict__ y, unsigned int *err)
{
    __shared__ Smem S;
    const int64_t ntiles = (n + kRows - 1) / kRows;
    if ((int64_t)blockIdx.x >= ntiles) return;
    tile_setup(S, params);
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * kRows + threadIdx.x;
        float f[kIn];
#pragma unroll
        for (int q = 0; q < kIn; ++q) f[q] = i < n ? x[i * kIn + q] : 0.f;
        store_features(S, f);
        float out[kOut];
        if (!forward_tile(S, phase, out)) {
            if (threadIdx.x == 0) atomicOr(err, 1u);
            break;
        }
        if (i < n) {
            y[i * kOut + 0] = out[0];
            y[i * kOut + 1] = out[1];
        }
    }
    tile_teardown(S);
}

constexpr int kTrainThreads = 256;
constexpr int kChunk = 64;                          // samples staged at once
constexpr int kPerThread = (kParams + kTrainThreads - 1) / kTrainThreads;   // 21

struct TrainSmem {
    float w[kParams];
    float x[kChunk][kIn];
    float h1[kChunk][kHid];
    float h2[kChunk][kHid];
    float d1[kChunk][kHid];   // dL/d(pre-activation of layer 1)
    float d2[kChunk][kHid];   // dL/d(pre-activation of layer 2)
    float dy[kChunk][kOut];
};

// the sample at position i of the order (a * i + c) mod n, a coprime with n
__device__ __forceinline__ int64_t order(int64_t i, int64_t n, uint64_t a, uint64_t c)
{
    return (int64_t)(((uint64_t)i * a + c) % (uint64_t)n);
}

// Gradient of the summed loss over samples [base, base + count) of the order
// (scaled by `scale`), added into grad; loss sums into loss[0..1].
__global__ void __launch_bounds__(kTrainThreads) grad_kernel(const float *__restrict__ params,
                                                             const float *__restrict__ feat,
                                                             const uint32_t *__restrict__ label, int64_t n,
                                                             int64_t base, int64_t count, uint64_t a, uint64_t c,
                                                             float tau, float scale, float *grad, double *loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) S.w[i] = params[i];
    float acc[kPerThread];
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) acc[q] = 0.f;
    float l0 = 0.f, l1 = 0.f;
    __syncthreads();
    const float *W1 = S.w + kOffW1, *B1 = S.w + kOffB1, *W2 = S.w + kOffW2, *B2 = S.w + kOffB2, *W3 = S.w + kOffW3,
                *B3 = S.w + kOffB3;
    const int64_t per = (count + gridDim.x - 1) / gridDim.x;
    const int64_t lo = min(count, per * (int64_t)blockIdx.x), hi = min(count, lo + per);
    for (int64_t c0 = lo; c0 < hi; c0 += kChunk) {
        const int m = (int)min((int64_t)kChunk, hi - c0);
        // forward and backward, one sample per thread (threads 0..m-1)
        if (threadIdx.x < m) {
            const int s = threadIdx.x;
            const int64_t idx = order(base + c0 + s, n, a, c);
            float x[kIn], h1[kHid];
#pragma unroll
            for (int q = 0; q < kIn; ++q) x[q] = S.x[s][q] = feat[idx * kIn + q];
            for (int j = 0; j < kHid; ++j) {
                float z = B1[j];
#pragma unroll
                for (int q = 0; q < kIn; ++q) z = fmaf(W1[j * kIn + q], x[q], z);
                h1[j] = fmaxf(z, 0.f);
                S.h1[s][j] = h1[j];
            }
            float y0 = B3[0], y1 = B3[1];
            for (int j = 0; j < kHid; ++j) {
                float z = B2[j];
                for (int q = 0; q < kHid; ++q) z = fmaf(W2[j * kHid + q], h1[q], z);
                const float h = fmaxf(z, 0.f);
                S.h2[s][j] = h;
                y0 = fmaf(W3[j], h, y0);
                y1 = fmaf(W3[kHid + j], h, y1);
            }
            const float t = log2f((float)min(max(label[idx], 1u), 64u));
            const float e0 = y0 - t, e1 = t - y1;
            l0 += e0 * e0;
            l1 += fmaxf(tau * e1, (tau - 1.f) * e1);
            const float g0 = 2.f * e0 * scale, g1 = (e1 > 0.f ? -tau : 1.f - tau) * scale;
            S.dy[s][0] = g0;
            S.dy[s][1] = g1;
            for (int j = 0; j < kHid; ++j)
                S.d2[s][j] = S.h2[s][j] > 0.f ? fmaf(W3[j], g0, W3[kHid + j] * g1) : 0.f;
            for (int q = 0; q < kHid; ++q) {
                float z = 0.f;
                for (int j = 0; j < kHid; ++j) z = fmaf(W2[j * kHid + q], S.d2[s][j], z);
                S.d1[s][q] = h1[q] > 0.f ? z : 0.f;
            }
        }
        __syncthreads();
        // parameter gradients: thread p owns parameters p, p + 256, ...
#pragma unroll
        for (int q = 0; q < kPerThread; ++q) {
            const int p = threadIdx.x + q * kTrainThreads;
            if (p >= kParams) break;
            float g = 0.f;
            if (p < kOffB1) {
                const int j = p / kIn, i = p % kIn;
                for (int s = 0; s < m; ++s) g = fmaf(S.d1[s][j], S.x[s][i], g);
            } else if (p < kOffW2) {
                const int j = p - kOffB1;
                for (int s = 0; s < m; ++s) g += S.d1[s][j];
            } else if (p < kOffB2) {
                const int j = (p - kOffW2) / kHid, i = (p - kOffW2) % kHid;
                for (int s = 0; s < m; ++s) g = fmaf(S.d2[s][j], S.h1[s][i], g);
            } else if (p < kOffW3) {
                const int j = p - kOffB2;
                for (int s = 0; s < m; ++s) g += S.d2[s][j];
            } else if (p < kOffB3) {
                const int o = (p - kOffW3) / kHid, i = (p - kOffW3) % kHid;
                for (int s = 0; s < m; ++s) g = fmaf(S.dy[s][o], S.h2[s][i], g);
            } else {
                const int o = p - kOffB3;
                for (int s = 0; s < m; ++s) g += S.dy[s][o];
            }
            acc[q] += g;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
        const int p = threadIdx.x + q * kTrainThreads;
        if (p < kParams && acc[q] != 0.f) atomicAdd(&grad[p], acc[q]);
    }
    // loss sums (threads that held samples)
    for (int o = 16; o; o >>= 1) {
        l0 += __shfl_xor_sync(0xFFFFFFFFu, l0, o);
        l1 += __shfl_xor_sync(0xFFFFFFFFu, l1, o);
    }
    if ((threadIdx.x & 31) == 0 && (l0 != 0.f || l1 != 0.f)) {
        atomicAdd(&loss[0], (double)l0);
        atomicAdd(&loss[1], (double)l1);
    }
}

__global__ void adam_kernel(float *params, float *grad, float *m, float *v, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    params[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    grad[p] = 0.f;
}

uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// a multiplier coprime with n for the sample order of one epoch
uint64_t order_mult(int64_t n, uint32_t seed, int epoch)
{
    uint64_t a = 1000003ull + 2ull * (((uint64_t)seed * 2654435761ull + (uint64_t)epoch * 40503ull) % 1000000ull);
    if (n <= 1) return 1;
    a %= (uint64_t)n;
    if (a == 0) a = 1;
    while (gcd64(a, (uint64_t)n) != 1) a = a + 1 < (uint64_t)n ? a + 1 : 1;
    return a;
}

size_t train_smem() { return sizeof(TrainSmem); }

int check_params(const float *params)
{
    for (int i = 0; i < kParams; ++i)
        if (!std::isfinite(params[i])) return set_error(SPR_ERR_INVALID_ARG, "parameter %d is not finite", i);
    return SPR_OK;
}

struct Scratch {
    DevBuf w, g, m, v, loss;
    void release(cudaStream_t s)
    {
        buf_free(w, s);
        buf_free(g, s);
        buf_free(m, s);
        buf_free(v, s);
        buf_free(loss, s);
    }
};

}  // namespace

extern "C" int spr_policy_forward(const float *params, const float *features, int64_t n, float *out, spr_stream stream)
{
    clear_error();
    if (!params || (n > 0 && (!features || !out)) || n < 0) return set_error(SPR_ERR_INVALID_ARG, "bad arguments");
    SPR_TRY(check_params(params));
    if (n == 0) return SPR_OK;
    cudaStream_t s = as_stream(stream);
    DevBuf w, err;
    int rc = buf_alloc(w, sizeof(float) * (kParams + 1), s);
    if (rc == SPR_OK) rc = buf_alloc(err, sizeof(unsigned int), s);
    if (rc == SPR_OK) {
        cudaError_t e = cudaMemcpyAsync(w.p, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) {
            const int64_t tiles = (n + kRows - 1) / kRows;
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 4 * device_sm_count()));
            forward_kernel<<<grid, kRows, 0, s>>>(w.as<float>(), features, n, out, err.as<unsigned int>());
            e = cudaGetLastError();
        }
        unsigned int h = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err.p, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "policy forward: %s", cudaGetErrorString(e));
        else if (h) rc = set_error(SPR_ERR_DEVICE_TIMEOUT, "a tensor-core wait timed out");
    }
    buf_free(w, s);
    buf_free(err, s);
    return rc;
}

extern "C" int spr_policy_grad(const float *params, const float *features, const uint32_t *labels, int64_t n, float tau,
                               float *grad, double *loss, spr_stream stream)
{
    clear_error();
    if (!params || !grad || n < 1 || !features || !labels) return set_error(SPR_ERR_INVALID_ARG, "bad arguments");
    SPR_TRY(check_params(params));
    cudaStream_t s = as_stream(stream);
    Scratch sc;
    int rc = SPR_OK;
    if ((rc = buf_alloc(sc.w, sizeof(float) * kParams, s)) || (rc = buf_alloc(sc.g, sizeof(float) * kParams, s)) ||
        (rc = buf_alloc(sc.loss, 2 * sizeof(double), s))) {
        sc.release(s);
        return rc;
    }
    cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem());
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.w.p, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.g.p, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.loss.p, 0, 2 * sizeof(double), s);
    if (e == cudaSuccess) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kChunk - 1) / kChunk, 2 * device_sm_count()));
        grad_kernel<<<grid, kTrainThreads, train_smem(), s>>>(sc.w.as<float>(), features, labels, n, 0, n, 1, 0, tau,
                                                             1.f / (float)n, sc.g.as<float>(), sc.loss.as<double>());
        e = cudaGetLastError();
    }
    double l[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, sc.g.p, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(l, sc.loss.p, sizeof l, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "policy gradient: %s", cudaGetErrorString(e));
    if (loss) {
        loss[0] = l[0] / (double)n;
        loss[1] = l[1] / (double)n;
    }
    sc.release(s);
    return rc;
}

extern "C" int spr_policy_train(const float *features, const uint32_t *labels, int64_t n, float *params,
                                const spr_train_desc *d, float *loss_per_epoch, spr_stream stream)
{
    clear_error();
    if (!features || !labels || !params || !d || n < 1) return set_error(SPR_ERR_INVALID_ARG, "bad arguments");
    if (d->epochs < 1 || d->batch < 1 || !(d->lr > 0.f) || !(d->beta1 >= 0.f && d->beta1 < 1.f) ||
        !(d->beta2 >= 0.f && d->beta2 < 1.f) || !(d->eps > 0.f) || !(d->tau > 0.f && d->tau < 1.f))
        return set_error(SPR_ERR_INVALID_ARG, "bad training settings");
    SPR_TRY(check_params(params));
    cudaStream_t s = as_stream(stream);
    Scratch sc;
    int rc = SPR_OK;
    if ((rc = buf_alloc(sc.w, sizeof(float) * kParams, s)) || (rc = buf_alloc(sc.g, sizeof(float) * kParams, s)) ||
        (rc = buf_alloc(sc.m, sizeof(float) * kParams, s)) || (rc = buf_alloc(sc.v, sizeof(float) * kParams, s)) ||
        (rc = buf_alloc(sc.loss, 2 * sizeof(double), s))) {
        sc.release(s);
        return rc;
    }
    cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem());
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.w.p, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.g.p, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.m.p, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.v.p, 0, sizeof(float) * kParams, s);
    const int64_t batch = std::min<int64_t>(d->batch, n);
    const int64_t steps = (n + batch - 1) / batch;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((batch + kChunk - 1) / kChunk, 2 * device_sm_count()));
    int64_t t = 0;
    for (int ep = 0; ep < d->epochs && e == cudaSuccess; ++ep) {
        const uint64_t a = order_mult(n, d->seed, ep);
        const uint64_t c = ((uint64_t)d->seed * 97ull + (uint64_t)ep * 7919ull) % (uint64_t)n;
        e = cudaMemsetAsync(sc.loss.p, 0, 2 * sizeof(double), s);
        for (int64_t st = 0; st < steps && e == cudaSuccess; ++st) {
            const int64_t base = st * batch, cnt = std::min<int64_t>(batch, n - base);
            grad_kernel<<<grid, kTrainThreads, train_smem(), s>>>(sc.w.as<float>(), features, labels, n, base, cnt, a,
                                                                 c, d->tau, 1.f / (float)cnt, sc.g.as<float>(),
                                                                 sc.loss.as<double>());
            ++t;
            const float c1 = 1.f - powf(d->beta1, (float)t), c2 = 1.f - powf(d->beta2, (float)t);
            adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(sc.w.as<float>(), sc.g.as<float>(), sc.m.as<float>(),
                                                              sc.v.as<float>(), d->lr, d->beta1, d->beta2, d->eps, c1,
                                                              c2);
            e = cudaGetLastError();
        }
        if (loss_per_epoch && e == cudaSuccess) {
            double l[2];
            e = cudaMemcpyAsync(l, sc.loss.p, sizeof l, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            loss_per_epoch[ep] = (float)(l[0] / (double)n);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(params, sc.w.p, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "policy training: %s", cudaGetErrorString(e));
    sc.release(s);
    return rc;
}
