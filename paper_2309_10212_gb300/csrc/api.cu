// api.cu -- error reporting, the pluggable device allocator and small
// helpers behind the C ABI.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "spr_common.cuh"

namespace spr {

namespace {
thread_local char g_err[512] = "";
spr_alloc_fn g_alloc = nullptr;
spr_free_fn g_free = nullptr;
void *g_ctx = nullptr;
std::mutex g_alloc_mu;
int g_sm_count = 0;
}  // namespace

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return status;
}

void clear_error() { g_err[0] = '\0'; }

void *dev_alloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 256;
    spr_alloc_fn a;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        ctx = g_ctx;
    }
    if (a) return a(bytes, reinterpret_cast<spr_stream>(s), ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s)
{
    if (!p) return;
    spr_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_ctx;
    }
    if (f) f(p, bytes, reinterpret_cast<spr_stream>(s), ctx);
    else cudaFree(p);
}

int buf_alloc(DevBuf &b, size_t bytes, cudaStream_t s)
{
    b.p = dev_alloc(bytes, s);
    if (!b.p) {
        b.bytes = 0;
        return set_error(SPR_ERR_OUT_OF_MEMORY, "device allocation of %zu bytes failed", bytes);
    }
    b.bytes = bytes;
    return SPR_OK;
}

void buf_free(DevBuf &b, cudaStream_t s)
{
    if (b.p) dev_free(b.p, b.bytes, s);
    b.p = nullptr;
    b.bytes = 0;
}

int buf_reserve(DevBuf &b, size_t bytes, cudaStream_t s)
{
    if (b.p && b.bytes >= bytes) return SPR_OK;
    if (b.p) {
        cudaStreamSynchronize(s);
        buf_free(b, s);
    }
    return buf_alloc(b, bytes, s);
}

int device_sm_count()
{
    if (g_sm_count == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        g_sm_count = n;
    }
    return g_sm_count;
}

}  // namespace spr

extern "C" const char *spr_last_error(void) { return spr::g_err; }

extern "C" const char *spr_status_string(int status)
{
    switch (status) {
    case SPR_OK: return "ok";
    case SPR_ERR_INVALID_ARG: return "invalid argument";
    case SPR_ERR_OUT_OF_MEMORY: return "out of device memory";
    case SPR_ERR_CACHE_TOO_SMALL: return "cache budget below 8 slots";
    case SPR_ERR_CUDA: return "CUDA runtime error";
    case SPR_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case SPR_ERR_NOT_CONVERGED: return "render did not converge within max_passes";
    case SPR_ERR_NOT_IMPLEMENTED: return "not implemented";
    case SPR_ERR_NO_DEVICE: return "no usable CUDA device";
    case SPR_ERR_DEVICE_ERROR: return "a kernel reported an internal error";
    default: return "unknown status";
    }
}

extern "C" int spr_version(void) { return 10000; }

extern "C" int spr_set_allocator(spr_alloc_fn alloc, spr_free_fn free_fn, void *ctx)
{
    spr::clear_error();
    if ((alloc == nullptr) != (free_fn == nullptr))
        return spr::set_error(SPR_ERR_INVALID_ARG, "alloc and free must both be set or both be NULL");
    std::lock_guard<std::mutex> lk(spr::g_alloc_mu);
    spr::g_alloc = alloc;
    spr::g_free = free_fn;
    spr::g_ctx = alloc ? ctx : nullptr;
    return SPR_OK;
}
