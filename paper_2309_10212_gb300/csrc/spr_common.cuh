// spr_common.cuh -- shared host/device helpers of the CUDA path.
//
// Error plumbing behind the C ABI, the pluggable device allocator, the
// volume descriptor, and the single-precision error-free transforms that
// make the traversal decisions of Sec. 3.3 exact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "spr.h"

namespace spr {

// ------------------------------------------------------------------ errors
int set_error(int status, const char *fmt, ...);
void clear_error();

#define SPR_CUDA_TRY(call)                                                         \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::spr::set_error(SPR_ERR_CUDA, "%s failed: %s (%s:%d)", #call,  \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)

#define SPR_TRY(call)                                                              \
    do {                                                                           \
        int s_ = (call);                                                           \
        if (s_ != SPR_OK) return s_;                                               \
    } while (0)

// ------------------------------------------------------------- allocation
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// an owning device buffer; the owner frees it explicitly (no destructors
// cross the C ABI)
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <class T> T *as() const { return static_cast<T *>(p); }
};
int buf_alloc(DevBuf &b, size_t bytes, cudaStream_t s);
void buf_free(DevBuf &b, cudaStream_t s);
// grow-only reallocation (contents are not kept)
int buf_reserve(DevBuf &b, size_t bytes, cudaStream_t s);

int device_sm_count();

inline cudaStream_t as_stream(spr_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------ volume
// Grid sizes: nb = ceil(D/4) compressed blocks, nc = ceil(nb/4) coarse cells;
// traversal uses tb = ceil((D-1)/4) blocks that own cells and tc = ceil(tb/4).
struct VolGeom {
    int32_t dims[3];
    int32_t nb[3], nc[3], tb[3], tc[3];
    int32_t rate;
    int64_t nblocks, ncoarse;
};

VolGeom make_geom(const int32_t dims[3], int rate);

}  // namespace spr

struct spr_volume {
    spr::VolGeom g;
    spr::DevBuf comp;     // nblocks * 8 * rate bytes
    spr::DevBuf fine;     // float2 per block
    spr::DevBuf coarse;   // float2 per coarse cell
    spr::DevBuf planes;   // uint8 per block: bit planes its parse reads (0: all-zero block)
};

// ======================================================== device arithmetic
namespace spr {

// Error-free transforms in single precision (Dekker, Knuth), written with
// explicit round-to-nearest intrinsics so that no contraction changes them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Exact sign of (a*b - c*d) for finite floats whose products neither
// overflow nor underflow: the four-term expansion p + pe - q - qe is grown
// term by term (Shewchuk's grow-expansion); its sign is the sign of its most
// significant nonzero component.
static __device__ __noinline__ int exact_sign_diff(float a, float b, float c, float d)
{
    float p, pe, q, qe;
    two_prod(a, b, p, pe);
    two_prod(c, d, q, qe);
    float e[4];
    int n = 1;
    e[0] = pe;
    float terms[3] = {-qe, -q, p};
    for (int t = 0; t < 3; ++t) {
        float Q = terms[t];
        for (int i = 0; i < n; ++i) {
            float s, h;
            two_sum(Q, e[i], s, h);
            e[i] = h;
            Q = s;
        }
        e[n++] = Q;
    }
    for (int i = 3; i >= 0; --i)
        if (e[i] != 0.0f) return e[i] > 0.0f ? 1 : -1;
    return 0;
}

// A ray parameter t = n / ad with ad > 0 (ad a direction magnitude, n a
// signed plane offset exact in single precision).
struct Tq {
    float n, ad;
};

// sign(t_a - t_b): a filtered exact comparison.  The single-precision
// difference decides whenever it exceeds its rounding bound; otherwise the
// exact expansion does.
__device__ __forceinline__ int tcmp(Tq a, Tq b)
{
    float p = __fmul_rn(a.n, b.ad), q = __fmul_rn(b.n, a.ad);
    float dd = __fsub_rn(p, q);
    float bound = __fmul_rn(__fadd_rn(fabsf(p), fabsf(q)), 3.0e-7f);
    if (dd > bound) return 1;
    if (dd < -bound) return -1;
    return exact_sign_diff(a.n, b.ad, b.n, a.ad);
}

// the ray of one pixel: eye, direction, |direction| and sign per axis
struct Ray {
    float e[3], d[3], ad[3];
    int sgn[3];
};

__device__ __forceinline__ void make_ray(Ray &r, const float eye[3], const float p00[3],
                                         const float du[3], const float dv[3], int px, int py)
{
    float fi = __fadd_rn((float)px, 0.5f), fj = __fadd_rn((float)py, 0.5f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float t2 = __fadd_rn(p00[a], __fmul_rn(fi, du[a]));
        float d = __fadd_rn(t2, __fmul_rn(fj, dv[a]));
        r.e[a] = eye[a];
        r.d[a] = d;
        r.ad[a] = fabsf(d);
        r.sgn[a] = (d > 0.0f) - (d < 0.0f);
    }
}

// crossing time of the plane {x_a = X}: n = (X - e_a) * sgn_a, exact
__device__ __forceinline__ Tq plane_t(const Ray &r, int a, float X)
{
    float n = __fsub_rn(X, r.e[a]);
    Tq t;
    t.n = r.sgn[a] > 0 ? n : -n;
    t.ad = r.ad[a];
    return t;
}

}  // namespace spr
