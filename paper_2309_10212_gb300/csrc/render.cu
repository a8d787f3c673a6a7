// render.cu -- the per-pass wavefront of the speculative progressive
// isosurface raycaster (Fig. 2, Sec. 3, 4) and the renderer part of the C ABI.
//
// One pass, all on the device, one host read of a small counter record:
//   traverse   (Sec. 3.3, 4.1) each live ray resumes its two-level walk
//              (coarse cells of 4^3 blocks, then blocks) and records its next
//              k visible blocks in R_BID at i*k + j; the visible block and its
//              +x/+y/+z neighbours are marked in two bitmaps (Sec. 3.4);
//   group      (Sec. 3.6, 4.2) the bitmaps compact to sorted lists I_BVis and
//              I_BAct; entries are counted per visible block, scanned into
//              O_BRays and scattered so each block's entries are contiguous;
//   cache      (Sec. 3.5) active blocks are looked up; misses take the least
//              recently used slots not needed by this pass;
//   decode     the misses are decompressed into their slots;
//   intersect  (Sec. 3.7, 4.3) each entry's ray is clipped to its block and
//              walked cell by cell; the first root of the trilinear cubic is
//              packed into a 64-bit key and atomicMin'ed per ray (Sec. 4.4);
//   resolve    hits and rays that left the volume are written out; the live
//              rays are compacted, in order, for the next pass.
// Traversal decisions use exact predicates (spr_common.cuh); intersection
// runs in block-local single precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "decode.cuh"
#include "kernels.cuh"
#include "scan.cuh"
#include "mlp.cuh"
#include "spr_common.cuh"

namespace spr {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint64_t kNoKey = ~0ull;
constexpr uint64_t kStep = 1;   // state flag: the saved block was already taken
constexpr uint64_t kDone = 2;   // state flag: the walk left the volume
// state flag set by ray generation: the saved block is where the ray enters
// the box of blocks that hold the isovalue, not where it enters the volume
// (the blocks before it hold nothing); cleared by the first walk
constexpr uint64_t kBoxed = 4;

// counter record, device resident, read by the host once per pass
enum Ctr {
    C_NVIS = 0,
    C_NACT,
    C_NENT,
    C_NMISS,
    C_NUNTOUCHED,
    C_NLIVE,
    C_OVERFLOW,
    C_EVICT,
    C_HIT,
    C_MISSRAY,
    C_SCANFLAGS,
    C_BAD,
    C_STEPS,     // walk steps of all rays this pass
    C_MAXSTEPS,  // longest walk this pass
    C_NEEDUSED,  // victims taken from the used-slot list (the rest are fresh slots)
    C_QISECT,    // work queue of the intersection: entries handed out
    C_KTOT,      // per-ray speculation: entries of the attempt (sum of the rays' k)
    C_COUNT = 20
};

// Per-ray speculation (modes SPR_SPEC_HASHED and SPR_SPEC_LEARNED): live
// position i takes kray[i] entries starting at koff[i] (an exclusive scan of
// kray), and every entry written records its position in eray.  With koff
// null every ray takes PassState::kk entries at i * kk.
struct Spec {
    const uint32_t *kray, *koff;
    uint32_t *eray;
};

// Training traces of the plain raycaster (spr_set_trace).  Per pass, live
// rays with hash(ray) mod `mod` == 0 append (features, ray, blocks taken so
// far); resolve keeps, per ray, the visible blocks taken (`taken`) and, when
// the ray finishes, how many it needed in all (`need`: up to and including
// the hit block, or every visible block of a miss).
struct Trace {
    float *feat;        // [cap][12]
    uint32_t *ray, *cons;
    uint32_t *count;    // samples appended (may pass cap; only cap are kept)
    uint32_t cap, mod;
    uint32_t *taken, *need;   // per ray
};


// The pass loop's state lives on the device, so that a pass (and a whole
// render, as one graph launch) needs no host round trip: begin_pass_kernel
// applies the speculation rule, end_pass_kernel records the pass, swaps the
// double-buffered lists, or halves k / the ray window when the pass overflowed
// the cache, and decides whether another pass runs.
struct PassState {
    uint32_t n_live;      // live rays at the start of the pass in progress
    uint32_t k, kk, nproc;  // rule's k, k of this attempt, live rays taken
    uint32_t pass;        // passes completed since ray generation
    uint32_t parity;      // bit 0: live list in use, bit 1: LRU list in use
    uint32_t retries;     // overflowed attempts of the pass in progress
    uint32_t open;        // 1 when an overflowed pass waits for its retry
    uint32_t max_passes;  // stop after this many passes
    uint32_t run;         // 1 while passes should continue
    uint32_t error;       // bit 0: wait timeout, bits 1..: kernel error flags
    uint32_t spec_mode, k_fixed, k_max;
    uint32_t npix;
    uint32_t n_enter;     // rays that entered the volume at ray generation
    uint32_t attempts;    // pass attempts since ray generation (retries included)
    // LRU cache: slots >= fresh_lo were never used (handed out in increasing
    // order, they are the least recently used); the used ones are listed, least
    // recently used first, in the list selected by parity bit 1
    uint32_t fresh_lo, fresh_hi, n_used;
    uint32_t live_words;  // ceil(n_live / 32): words of the alive bitmap of this pass
    uint32_t coop_below;  // passes with fewer live rays walk one ray per warp
    uint32_t seg_threads; // lanes the segmented walk may use (0: off); see traverse_seg_kernel
    unsigned long long tot_decoded, tot_entries, tot_evicted, tot_hits;
};

struct Cam {
    float eye[3], p00[3], du[3], dv[3];
};

// every slot fresh again, the used-slot lists empty
__device__ __forceinline__ void lru_reset(PassState *ps)
{
    ps->fresh_lo = ps->fresh_hi = 0;
    ps->n_used = 0;
}

// Per-render parameters in device memory, copied from a pinned host block by
// the first node of the render's start graph (so the captured graphs stay
// valid when the camera, isovalue, speculation or pass limit change).
// one view of a batch: its camera and isovalue
struct View {
    Cam cam;
    float iso;
};
constexpr int kMaxViews = 64;

struct DevParams {
    uint32_t spec_mode, k_fixed, k_max, npix;
    uint32_t more;    // passes this call may run
    uint32_t reset;   // 1: empty the cache before ray generation
    uint32_t coop_below;
    uint32_t seg_threads;
    uint32_t n_views;
    View views[kMaxViews];   // the first n_views are copied
};

// occupancy of the three skipping levels for the current isovalue: one bit
// per block (fine), per 4^3 blocks (coarse) and per 16^3 blocks (super)
// Brick masks: fmask[c] has bit x+4y+16z set when block 4c+(x,y,z) of coarse
// cell c holds the isovalue in its fine range; smask[s] has bit x+4y+16z set
// when coarse cell 4s+(x,y,z) of super cell s has a nonzero fmask.  A walk
// loads one word when it enters a coarse or super cell and then steps through
// that cell's blocks without touching memory.
//
// The occupied box of a view: the lowest and highest block index per axis
// among the blocks that hold its isovalue, {lo x, y, z, -, hi x, y, z, -}
// (lo > hi when no block does).  A ray meets a visible block only while it
// is inside the box, so its walk starts where it enters the box and ends
// where it leaves it.
struct Occ {
    const unsigned long long *fmask, *smask;
    const int *box;   // 8 ints per view
    int ns[3];   // super grid over the coarse grid: ceil(nc / 4)
    int ts[3];   // super cells the traversal can visit: ceil(tc / 4)
};

// bit i (0..63) of a 64-bit brick mask, read from its 32-bit half
__device__ __forceinline__ bool mask_bit(unsigned long long m, int i)
{
    const uint32_t h = (i & 32) ? (uint32_t)(m >> 32) : (uint32_t)m;
    return (h >> (i & 31)) & 1u;
}

// A walk has passed the occupied box once a block index goes beyond the
// box's last index in the walk's direction (indices change monotonically, so
// no later block is in the box): sgn_a * b_a > lim_a with lim_a = hi_a for
// sgn_a > 0, -lo_a for sgn_a < 0 and INT_MAX for sgn_a = 0.
__device__ __forceinline__ void box_limits(const int sgn[3], const int *bx, int lim[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) lim[a] = sgn[a] > 0 ? bx[4 + a] : (sgn[a] < 0 ? -bx[a] : INT_MAX);
}

__device__ __forceinline__ bool past_box(const int b[3], const int sgn[3], const int lim[3])
{
    return sgn[0] * b[0] > lim[0] || sgn[1] * b[1] > lim[1] || sgn[2] * b[2] > lim[2];
}

// camera and isovalue live in device memory (read at kernel start), so that a
// captured pass graph stays valid when they change
struct Geo {
    VolGeom g;
    const float2 *fine;
    const float2 *coarse;
    const View *views;     // n_views records (device)
    int W, H;
    int64_t WH;            // pixels per view; ray id = view * WH + y * W + x
    int64_t fstride, sstride;   // brick-mask words per view (coarse, super)
    Occ occ;
};

// the view and pixel of a ray id
__device__ __forceinline__ void ray_pixel(const Geo &P, uint32_t ray, int &view, int &px, int &py)
{
    const uint32_t v = (uint32_t)(ray / (uint64_t)P.WH);
    const uint32_t p = ray - v * (uint32_t)P.WH;
    view = (int)v;
    px = (int)(p % (uint32_t)P.W);
    py = (int)(p / (uint32_t)P.W);
}



__device__ __forceinline__ bool holds(float2 r, float iso) { return r.x <= iso && iso <= r.y; }

__device__ __forceinline__ uint64_t pack_state(const int b[3], uint64_t flags)
{
    return (uint64_t)(b[0] & 0xFFFF) | ((uint64_t)(b[1] & 0xFFFF) << 16) |
           ((uint64_t)(b[2] & 0xFFFF) << 32) | (flags << 48);
}

// ---------------------------------------------------------- exact walking
// A walk through the block grid.  Per axis it keeps the exact signed offset N
// of the next block plane (so t = N / |d|) and t itself rounded to single
// precision (relative error below 2 ulps).  The next crossing is decided on
// the rounded t; when two axes lie within 5e-7 of each other, which contains
// every case where rounding could swap them, the exact comparison decides.
struct Walk {
    Ray r;
    float inv[3];   // 1 / |d_a|
    int b[3];       // current block
    float N[3], t[3];
};

__device__ __forceinline__ void set_axis(Walk &w, const VolGeom &g, int a)
{
    if (w.r.sgn[a] == 0) {
        w.N[a] = 0.f;
        w.t[a] = INFINITY;
        return;
    }
    float X = w.r.sgn[a] > 0 ? (float)min(4 * (w.b[a] + 1), g.dims[a] - 1) : (float)(4 * w.b[a]);
    float n = __fsub_rn(X, w.r.e[a]);
    w.N[a] = w.r.sgn[a] > 0 ? n : -n;
    w.t[a] = __fmul_rn(w.N[a], w.inv[a]);
}

__device__ __forceinline__ void walk_init(Walk &w, const VolGeom &g)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.inv[a] = w.r.sgn[a] ? __frcp_rn(w.r.ad[a]) : 0.f;
        set_axis(w, g, a);
    }
}

// the set of axes whose plane (offsets N, rounded times t) is crossed first
__device__ __forceinline__ int first_axes(const float t[3], const float N[3], const float ad[3])
{
    float m = fminf(fminf(t[0], t[1]), t[2]);
    float thr = m + fabsf(m) * 5e-7f;
    int mask = (t[0] <= thr) | ((t[1] <= thr) << 1) | ((t[2] <= thr) << 2);
    if (__popc(mask) > 1) {
        int out = 0;
        Tq best{0.f, 1.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!(mask >> a & 1)) continue;
            Tq ta{N[a], ad[a]};
            int c = out ? tcmp(ta, best) : -1;
            if (c < 0) {
                best = ta;
                out = 1 << a;
            } else if (c == 0) {
                out |= 1 << a;
            }
        }
        mask = out;
    }
    return mask;
}

// step to the next block; false when the walk leaves the traversal grid
__device__ __forceinline__ bool walk_step(Walk &w, const VolGeom &g)
{
    int mask = first_axes(w.t, w.N, w.r.ad);
    bool ok = mask != 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (mask >> a & 1) {
            w.b[a] += w.r.sgn[a];
            if (w.b[a] < 0 || w.b[a] >= g.tb[a]) ok = false;
            else set_axis(w, g, a);
        }
    return ok;
}

// sign(t_X - T) for a plane X on axis a, filtered on the rounded times
__device__ __forceinline__ int cmp_plane(const Walk &w, int a, float X, Tq T, float Tv)
{
    float n = __fsub_rn(X, w.r.e[a]);
    Tq tx{w.r.sgn[a] > 0 ? n : -n, w.r.ad[a]};
    float tv = __fmul_rn(tx.n, w.inv[a]);
    float d = tv - Tv, tol = (fabsf(tv) + fabsf(Tv)) * 3e-7f;
    if (d > tol) return 1;
    if (d < -tol) return -1;
    return exact_sign_diff(tx.n, T.ad, T.n, tx.ad);
}

// block index along axis a containing p(T+), known to lie in [lo, hi].  The
// single-precision position p = e + T d is within tol of the true one; when
// it is farther than tol from every block plane its floor is certain,
// otherwise exact plane tests decide.
__device__ __forceinline__ int locate_in(const Walk &w, int a, Tq T, float Tv, int lo, int hi)
{
    float p = fmaf(Tv, w.r.d[a], w.r.e[a]);
    float q = fminf(fmaxf(__fmul_rn(p, 0.25f), (float)lo - 1.f), (float)hi + 1.f);
    {
        float fq = floorf(q), frac = q - fq;
        float tol = (fabsf(Tv * w.r.d[a]) + fabsf(w.r.e[a])) * 1e-6f + 1e-6f;
        int b = (int)fq;
        if (frac > tol && frac < 1.f - tol && b >= lo && b <= hi) return b;
    }
    int b;
    if (w.r.sgn[a] > 0) {
        b = min(max((int)floorf(q), lo), hi);
        while (b + 1 <= hi && cmp_plane(w, a, (float)(4 * (b + 1)), T, Tv) <= 0) ++b;
        while (b - 1 >= lo && cmp_plane(w, a, (float)(4 * b), T, Tv) > 0) --b;
    } else {
        b = min(max((int)ceilf(q) - 1, lo), hi);
        while (b - 1 >= lo && cmp_plane(w, a, (float)(4 * b), T, Tv) <= 0) --b;
        while (b + 1 <= hi && cmp_plane(w, a, (float)(4 * (b + 1)), T, Tv) > 0) ++b;
    }
    return b;
}

// Leave the current level cell (sb blocks per side: 4 for coarse cells, 16
// for super cells; tl cells per axis).  The new block is the one containing
// the ray just after the exit point; false when the ray leaves the volume.
__device__ __forceinline__ bool skip_level(Walk &w, const VolGeom &g, int sb, const int tl[3])
{
    const int L = 4 * sb;
    const int lsb = sb == 16 ? 4 : 2;
    int c[3];
    float NL[3], TL[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c[a] = w.b[a] >> lsb;
        if (w.r.sgn[a] == 0) {
            NL[a] = 0.f;
            TL[a] = INFINITY;
            continue;
        }
        float X = w.r.sgn[a] > 0 ? (float)min(L * (c[a] + 1), g.dims[a] - 1) : (float)(L * c[a]);
        float n = __fsub_rn(X, w.r.e[a]);
        NL[a] = w.r.sgn[a] > 0 ? n : -n;
        TL[a] = __fmul_rn(NL[a], w.inv[a]);
    }
    int mask = first_axes(TL, NL, w.r.ad);
    if (!mask) return false;
    // the exit time, taken from the lowest axis of the set (static indexing)
    Tq T;
    float Tv;
    if (mask & 1) {
        T = Tq{NL[0], w.r.ad[0]};
        Tv = TL[0];
    } else if (mask & 2) {
        T = Tq{NL[1], w.r.ad[1]};
        Tv = TL[1];
    } else {
        T = Tq{NL[2], w.r.ad[2]};
        Tv = TL[2];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (mask >> a & 1) {
            c[a] += w.r.sgn[a];
            if (c[a] < 0 || c[a] >= tl[a]) return false;
            w.b[a] = w.r.sgn[a] > 0 ? sb * c[a] : min(sb * c[a] + sb - 1, g.tb[a] - 1);
        } else if (w.r.sgn[a] > 0) {
            w.b[a] = locate_in(w, a, T, Tv, w.b[a], min(sb * c[a] + sb - 1, g.tb[a] - 1));
        } else if (w.r.sgn[a] < 0) {
            w.b[a] = locate_in(w, a, T, Tv, sb * c[a], w.b[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) set_axis(w, g, a);
    return true;
}

// block index along axis a that contains p(T+)
__device__ int locate_block(const Ray &r, int a, Tq T, int tb)
{
    if (r.sgn[a] == 0) {
        float f = floorf(__fmul_rn(r.e[a], 0.25f));
        f = fminf(fmaxf(f, 0.f), (float)(tb - 1));
        return (int)f;
    }
    float p = fmaf(__fdiv_rn(T.n, T.ad), r.d[a], r.e[a]);
    float q = fminf(fmaxf(__fmul_rn(p, 0.25f), -1.f), (float)tb);
    int b;
    if (r.sgn[a] > 0) {
        b = min(max((int)floorf(q), 0), tb - 1);
        while (b + 1 <= tb - 1 && tcmp(plane_t(r, a, (float)(4 * (b + 1))), T) <= 0) ++b;
        while (b >= 1 && tcmp(plane_t(r, a, (float)(4 * b)), T) > 0) --b;
    } else {
        b = min(max((int)ceilf(q) - 1, 0), tb - 1);
        while (b >= 1 && tcmp(plane_t(r, a, (float)(4 * b)), T) <= 0) --b;
        while (b + 1 <= tb - 1 && tcmp(plane_t(r, a, (float)(4 * (b + 1))), T) > 0) ++b;
    }
    return b;
}

__device__ __forceinline__ void set_bit(uint32_t *bits, uint32_t b)
{
    atomicOr(bits + (b >> 5), 1u << (b & 31));   // result unused: a reduction
}

// A warp takes the next 32 items of a work queue (all lanes get the base).
// The intersection runs one wave of CTAs that loop until the queue is dry,
// so blocks with many entries do not hold back a fixed share of the grid.
// (The traversal keeps a grid-stride loop over several waves: its lanes
// diverge so much that a warp-wide take would wait on the longest ray.)
__device__ __forceinline__ uint32_t warp_take(uint32_t *q)
{
    uint32_t base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(q, 32u);
    return __shfl_sync(0xFFFFFFFFu, base, 0);
}

__device__ __forceinline__ void warp_add(uint32_t *ctr, uint32_t v)
{
    unsigned m = __activemask();
    uint32_t s = __reduce_add_sync(m, v);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(m) - 1) && s) atomicAdd(ctr, s);
}

// ------------------------------------------------------------- occupancy
// one thread per coarse cell: the bits of its 4^3 blocks
// and the occupied box: at launch box (8 ints) holds lo values above every
// block index and hi values of -1; blockDim is a multiple of 32
__global__ void fmask_kernel(const float2 *__restrict__ fine, VolGeom g, float iso,
                             unsigned long long *__restrict__ fmask, int *box)
{
    __shared__ int s_box[6];
    if (threadIdx.x < 6) s_box[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : -1;
    __syncthreads();
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncoarse;
         c += (int64_t)gridDim.x * blockDim.x) {
        int cx = (int)(c % g.nc[0]), cy = (int)((c / g.nc[0]) % g.nc[1]), cz = (int)(c / ((int64_t)g.nc[0] * g.nc[1]));
        unsigned long long m = 0ull;
        for (int k = 0; k < 64; ++k) {
            int x = 4 * cx + (k & 3), y = 4 * cy + ((k >> 2) & 3), z = 4 * cz + (k >> 4);
            if (x < g.nb[0] && y < g.nb[1] && z < g.nb[2] &&
                holds(fine[x + (int64_t)g.nb[0] * (y + (int64_t)g.nb[1] * z)], iso)) {
                m |= 1ull << k;
                lo[0] = min(lo[0], x);
                lo[1] = min(lo[1], y);
                lo[2] = min(lo[2], z);
                hi[0] = max(hi[0], x);
                hi[1] = max(hi[1], y);
                hi[2] = max(hi[2], z);
            }
        }
        fmask[c] = m;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int l = __reduce_min_sync(0xFFFFFFFFu, lo[a]), h = __reduce_max_sync(0xFFFFFFFFu, hi[a]);
        if ((threadIdx.x & 31) == 0 && h >= 0) {
            atomicMin(&s_box[a], l);
            atomicMax(&s_box[3 + a], h);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3 && s_box[3 + threadIdx.x] >= 0) {
        atomicMin(box + threadIdx.x, s_box[threadIdx.x]);
        atomicMax(box + 4 + threadIdx.x, s_box[3 + threadIdx.x]);
    }
}

// one thread per super cell: which of its 4^3 coarse cells hold any block
__global__ void smask_kernel(const unsigned long long *__restrict__ fmask, VolGeom g, Occ o,
                             unsigned long long *__restrict__ smask)
{
    const int64_t n = (int64_t)o.ns[0] * o.ns[1] * o.ns[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int sx = (int)(i % o.ns[0]), sy = (int)((i / o.ns[0]) % o.ns[1]), sz = (int)(i / ((int64_t)o.ns[0] * o.ns[1]));
        unsigned long long m = 0ull;
        for (int k = 0; k < 64; ++k) {
            int x = 4 * sx + (k & 3), y = 4 * sy + ((k >> 2) & 3), z = 4 * sz + (k >> 4);
            if (x < g.nc[0] && y < g.nc[1] && z < g.nc[2] &&
                fmask[x + (int64_t)g.nc[0] * (y + (int64_t)g.nc[1] * z)])
                m |= 1ull << k;
        }
        smask[i] = m;
    }
}

// ------------------------------------------------------------- ray setup
// Rays are enumerated in tiles of 8x4 pixels (a warp's worth), tiles in
// row-major order, so the rays one warp traverses and intersects are screen
// neighbours.  The live lists keep this order from pass to pass.
constexpr int kRayTileW = 8, kRayTileH = 4;

__host__ __device__ inline int64_t tiled_ray_count(int W, int H)
{
    return (int64_t)((W + kRayTileW - 1) / kRayTileW) * ((H + kRayTileH - 1) / kRayTileH) * 32;
}

// pixel of tiled position t, or -1 where the tile overhangs the image
__device__ __forceinline__ int64_t tiled_pixel(int64_t t, int W, int H)
{
    const int64_t tile = t >> 5;
    const int l = (int)(t & 31);
    const int tiles_x = (W + kRayTileW - 1) / kRayTileW;
    const int x = (int)(tile % tiles_x) * kRayTileW + (l & (kRayTileW - 1));
    const int y = (int)(tile / tiles_x) * kRayTileH + (l >> 3);
    return (x < W && y < H) ? (int64_t)y * W + x : -1;
}

// Ray generation, one thread per tiled position: clear the pixel's outputs,
// find the ray's entry block, and set bit t of `enter` (warp ballots) when
// the ray enters the domain.
__global__ void __launch_bounds__(256) raygen_kernel(Geo P, int H, uint64_t *__restrict__ state,
                                                     uint8_t *__restrict__ status, uint64_t *__restrict__ keys,
                                                     float *__restrict__ depth, uint32_t *__restrict__ rgba,
                                                     uint32_t *__restrict__ block, uint64_t *__restrict__ cell,
                                                     int32_t *__restrict__ final_pass, uint32_t *__restrict__ enter,
                                                     int64_t n_tiled, PassState *ps, const uint32_t *lru_reset_flag,
                                                     const uint32_t *n_views_dev, uint32_t n_views_host)
{
    if (lru_reset_flag && blockIdx.x == 0 && threadIdx.x == 0 && *lru_reset_flag) lru_reset(ps);
    const VolGeom &g = P.g;
    const int64_t tpv = tiled_ray_count(P.W, H);   // tiled positions per view
    // views at or beyond the active count (a renderer sized for more views)
    // generate no rays and leave their pixels untouched
    const int64_t n_act = (int64_t)(n_views_dev ? *n_views_dev : n_views_host) * tpv;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiled;
         t += (int64_t)gridDim.x * blockDim.x) {   // n_tiled is a multiple of 32: whole warps iterate
        const int64_t view = t / tpv;
        const int64_t pv = t < n_act ? tiled_pixel(t - view * tpv, P.W, H) : -1;
        bool in = false;
        if (pv >= 0) {
            const int64_t p = view * P.WH + pv;   // ray id
            const Cam &cam = P.views[view].cam;
            keys[p] = kNoKey;
            depth[p] = INFINITY;
            rgba[p] = 0u;
            block[p] = kNone;
            cell[p] = kNoKey;
            final_pass[p] = 0;
            Ray r;
            make_ray(r, cam.eye, cam.p00, cam.du, cam.dv, (int)(pv % P.W), (int)(pv / P.W));
            Tq tin{0.f, 1.f}, tout{0.f, 1.f};
            bool have_out = false, outside = false;
            for (int a = 0; a < 3; ++a) {
                if (r.sgn[a] == 0) {
                    if (r.e[a] < 0.f || r.e[a] > (float)(g.dims[a] - 1)) outside = true;
                    continue;
                }
                float nearp = r.sgn[a] > 0 ? 0.f : (float)(g.dims[a] - 1);
                float farp = r.sgn[a] > 0 ? (float)(g.dims[a] - 1) : 0.f;
                Tq tn = plane_t(r, a, nearp), tf = plane_t(r, a, farp);
                if (tcmp(tn, tin) > 0) tin = tn;
                if (!have_out || tcmp(tf, tout) < 0) {
                    tout = tf;
                    have_out = true;
                }
            }
            if (outside || !have_out || tcmp(tin, tout) >= 0) {
                status[p] = 2;
            } else {
                int b[3];
                for (int a = 0; a < 3; ++a) b[a] = locate_block(r, a, tin, g.tb[a]);
                // the part of the ray inside the occupied box: per axis the
                // blocks lo..hi are those the ray is in for t in [t(near), t(far))
                const int *bx = P.occ.box + 8 * view;
                Tq t0 = tin, t1 = tout;
                bool none = false, moved = false;
                for (int a = 0; a < 3; ++a) {
                    const int lo = bx[a], hi = bx[4 + a];
                    if (lo > hi || (r.sgn[a] == 0 && (b[a] < lo || b[a] > hi))) {
                        none = true;
                        break;
                    }
                    if (r.sgn[a] == 0) continue;
                    const Tq tn = plane_t(r, a, (float)(r.sgn[a] > 0 ? 4 * lo : 4 * (hi + 1)));
                    const Tq tf = plane_t(r, a, (float)(r.sgn[a] > 0 ? 4 * (hi + 1) : 4 * lo));
                    if (tcmp(tn, t0) > 0) {
                        t0 = tn;
                        moved = true;
                    }
                    if (tcmp(tf, t1) < 0) t1 = tf;
                }
                // a ray that misses the box stays live with its walk done,
                // so the live count (and the speculation it sets) is unchanged
                uint64_t fl = 0;
                if (none || tcmp(t0, t1) >= 0) {
                    fl = kDone;
                } else if (moved) {
                    for (int a = 0; a < 3; ++a) b[a] = locate_block(r, a, t0, g.tb[a]);
                    fl = kBoxed;
                }
                state[p] = pack_state(b, fl);
                status[p] = 0;
                in = true;
            }
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, in);
        if ((threadIdx.x & 31) == 0) enter[t >> 5] = bits;
    }
}

// one item per bit of a bitmap (compactions driven by ballot bitmaps)
struct BitCount {
    const uint32_t *bits;
    const uint32_t *skip;
    __device__ bool enabled() const { return !skip || !*skip; }
    __device__ uint32_t operator()(int64_t i) const { return (bits[i >> 5] >> (i & 31)) & 1u; }
};

// live list 0 from the enter bitmap: tiled position t -> its ray id
struct EnterEmit {
    uint32_t *out;
    int W, H;
    int64_t WH;
    __device__ void operator()(int64_t t, uint32_t pre, uint32_t c) const
    {
        if (!c) return;
        const int64_t tpv = tiled_ray_count(W, H), view = t / tpv;
        out[pre] = (uint32_t)(view * WH + tiled_pixel(t - view * tpv, W, H));
    }
};


// ------------------------------------------------------------- traversal
// Passes with fewer live rays than PassState::coop_below (default 16384, set
// with spr_set_warp_walk_threshold) walk one ray per warp
// (traverse_coop_kernel); larger passes one ray per thread (traverse_kernel).
constexpr uint32_t kCoopBelowDefault = 16384;
// lanes of the segmented walk (traverse_seg_kernel): a pass of n live rays
// gives each ray seg_threads / n lanes (a power of two up to 32, used from 2)
constexpr uint32_t kSegThreadsDefault = 262144;   // measured best of 0, 2^18 .. 2^21 (paper scale, medium)

// lanes per ray of this pass (1: the segmented walk is not used)
__device__ __forceinline__ int seg_lanes(const PassState *ps)
{
    const uint32_t n = ps->nproc, budget = ps->seg_threads;
    if (!budget || !n || budget / n < 2) return 1;
    const uint32_t q = min(budget / n, 32u);
    return 1 << (31 - __clz(q));
}

constexpr uint32_t kHalfWarpFrom = 4096;   // warp walks: a half warp per ray from this many rays

__global__ void __launch_bounds__(128) traverse_kernel(Geo P, const uint32_t *__restrict__ live0,
                                                       const uint32_t *__restrict__ live1,
                                                       const PassState *__restrict__ ps,
                                                       const uint64_t *__restrict__ state_in,
                                                       uint64_t *__restrict__ state_out,
                                                       uint32_t *__restrict__ rbid,
                                                       uint32_t *vis_bits, uint32_t *act_bits,
                                                       uint32_t *ctr, Spec S)
{
    const VolGeom &g = P.g;
    const uint32_t nproc = ps->nproc;
    if (nproc < ps->coop_below) return;   // few rays: traverse_coop_kernel walks them
    if (seg_lanes(ps) > 1) return;        // traverse_seg_kernel walks them
    const int kk = (int)ps->kk;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    // every step moves at least one block index monotonically, so a walk
    // never takes more steps than this; exceeding it is an internal error
    const int max_steps = 2 * (g.tb[0] + g.tb[1] + g.tb[2]) + 8;
    const uint32_t nb0 = g.nb[0], nb1 = g.nb[1], nc0 = g.nc[0], nc1 = g.nc[1];
    const uint32_t ns0 = P.occ.ns[0], ns1 = P.occ.ns[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nproc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t ray = live[i];
        Walk w;
        int view, px, py;
        ray_pixel(P, ray, view, px, py);
        {
            const Cam &cam = P.views[view].cam;
            make_ray(w.r, cam.eye, cam.p00, cam.du, cam.dv, px, py);
        }
        const unsigned long long *fm = P.occ.fmask + view * P.fstride, *sm = P.occ.smask + view * P.sstride;
        const uint64_t st = state_in[ray];
        w.b[0] = (int)(st & 0xFFFF);
        w.b[1] = (int)((st >> 16) & 0xFFFF);
        w.b[2] = (int)((st >> 32) & 0xFFFF);
        uint64_t flags = st >> 48;
        const uint64_t off = S.koff ? S.koff[i] : (uint64_t)i * kk;
        const int ki = S.koff ? (int)S.kray[i] : kk;
        uint32_t *out = rbid + off;
        int cnt = 0;
        bool alive = !(flags & kDone);
        if (alive) {
            walk_init(w, g);
            if (flags & kStep) alive = walk_step(w, g);
        }
        flags &= ~(kStep | kBoxed);
        int lim[3];
        box_limits(w.r.sgn, P.occ.box + 8 * view, lim);
        int steps = 0;
        uint32_t cur_s = 0xFFFFFFFFu, cur_c = 0xFFFFFFFFu;
        unsigned long long smask = 0ull, fmask = 0ull;
        while (alive) {
            if (++steps > max_steps) {
                atomicOr(&ctr[C_BAD], 2u);
                alive = false;
                break;
            }
            const int *b = w.b;
            if (past_box(b, w.r.sgn, lim)) {
                alive = false;
                break;
            }
            uint32_t sc = (uint32_t)(b[0] >> 4) + ns0 * ((uint32_t)(b[1] >> 4) + ns1 * (uint32_t)(b[2] >> 4));
            if (sc != cur_s) {
                smask = __ldg(sm + sc);
                cur_s = sc;
            }
            if (!mask_bit(smask, ((b[0] >> 2) & 3) + 4 * ((b[1] >> 2) & 3) + 16 * ((b[2] >> 2) & 3))) {
                alive = skip_level(w, g, smask ? 4 : 16, smask ? g.tc : P.occ.ts);
                continue;
            }
            uint32_t c = (uint32_t)(b[0] >> 2) + nc0 * ((uint32_t)(b[1] >> 2) + nc1 * (uint32_t)(b[2] >> 2));
            if (c != cur_c) {
                fmask = __ldg(fm + c);
                cur_c = c;
            }
            if (mask_bit(fmask, (b[0] & 3) + 4 * (b[1] & 3) + 16 * (b[2] & 3))) {
                uint32_t blin = (uint32_t)b[0] + nb0 * ((uint32_t)b[1] + nb1 * (uint32_t)b[2]);
                if (S.eray) S.eray[off + cnt] = (uint32_t)i;
                out[cnt++] = blin;
                set_bit(vis_bits, blin);
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    int x = b[0] + (o & 1), y = b[1] + ((o >> 1) & 1), z = b[2] + (o >> 2);
                    if (x < g.nb[0] && y < g.nb[1] && z < g.nb[2])
                        set_bit(act_bits, (uint32_t)x + nb0 * ((uint32_t)y + nb1 * (uint32_t)z));
                }
                if (cnt == ki) {
                    flags |= kStep;
                    break;
                }
            }
            alive = walk_step(w, g);
        }
        if (!alive) flags |= kDone;
        for (int j = cnt; j < ki; ++j) out[j] = kNone;
        state_out[ray] = pack_state(w.b, flags);
        warp_add(&ctr[C_STEPS], (uint32_t)steps);
        {
            unsigned m = __activemask();
            uint32_t mx = __reduce_max_sync(m, (uint32_t)steps);
            if ((threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicMax(&ctr[C_MAXSTEPS], mx);
        }
    }
}

// One ray per warp or half warp, for passes whose few rays make the walk
// latency-bound.
// The walk is the same as traverse_kernel's; inside an occupied coarse cell
// the blocks are found in one step instead of one by one.  Lane 4a + k - 1
// (a < 3, k = 1..4) takes the k-th block-plane crossing of the ray along
// axis a inside the cell; the last crossing per axis leaves the cell or the
// volume, and the first of those, T_exit, ends the cell.  Exact comparisons
// with the other axes' crossings give each crossing the number of crossings
// per axis up to its time (the block after it) and its rank among the
// distinct times; crossings at one time from several axes are one
// (diagonal) step, represented by the lowest axis, as in walk_step.  The
// visible blocks of the cell are then taken in rank order, and the walk moves
// to the block after T_exit.  Empty coarse and super cells are skipped with
// skip_level, computed identically by all lanes.
template <int LPR>
__global__ void __launch_bounds__(128) traverse_coop_kernel(Geo P, const uint32_t *__restrict__ live0,
                                                            const uint32_t *__restrict__ live1,
                                                            const PassState *__restrict__ ps,
                                                            const uint64_t *__restrict__ state_in,
                                                            uint64_t *__restrict__ state_out,
                                                            uint32_t *__restrict__ rbid,
                                                            uint32_t *vis_bits, uint32_t *act_bits,
                                                            uint32_t *ctr, Spec S)
{
    static_assert(LPR == 16 || LPR == 32, "16 or 32 lanes per ray");
    const VolGeom &g = P.g;
    const uint32_t nproc = ps->nproc;
    if (nproc >= ps->coop_below) return;
    if (seg_lanes(ps) > 1) return;        // traverse_seg_kernel walks them
    // a half warp per ray when there are enough rays to fill the GPU (the
    // walk is then bound by instruction throughput), a whole warp per ray
    // for the last few (bound by each walk's latency)
    if ((LPR == 16) != (nproc >= kHalfWarpFrom)) return;
    const int kk = (int)ps->kk;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    const int max_steps = 2 * (g.tb[0] + g.tb[1] + g.tb[2]) + 8;
    const uint32_t nb0 = g.nb[0], nb1 = g.nb[1], nc0 = g.nc[0], nc1 = g.nc[1];
    const uint32_t ns0 = P.occ.ns[0], ns1 = P.occ.ns[1];
    // LPR lanes walk one ray: lanes 0-11 of the group take the crossings,
    // lane LPR - 1 the current block; masks, ballots and shuffles stay within
    // the group, so the two rays of a warp (LPR = 16) proceed independently
    constexpr int kShift = LPR == 16 ? 4 : 5;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LPR - 1);                   // lane within the group
    const int gshift = LPR == 16 ? (lane & 16) : 0;    // the group's first lane
    const unsigned full = LPR == 16 ? (0xFFFFu << gshift) : 0xFFFFFFFFu;
    const bool elane = gl < 12;
    const int ea = elane ? gl >> 2 : 0;     // axis of this lane's crossing
    const int ek = (gl & 3) + 1;            // its number along that axis
    uint32_t tot_steps = 0, max_seen = 0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> kShift; i < nproc;
         i += ((int64_t)gridDim.x * blockDim.x) >> kShift) {
        const uint32_t ray = live[i];
        Walk w;
        int view, px, py;
        ray_pixel(P, ray, view, px, py);
        {
            const Cam &cam = P.views[view].cam;
            make_ray(w.r, cam.eye, cam.p00, cam.du, cam.dv, px, py);
        }
        const unsigned long long *fm = P.occ.fmask + view * P.fstride, *sm = P.occ.smask + view * P.sstride;
        const uint64_t st = state_in[ray];
        w.b[0] = (int)(st & 0xFFFF);
        w.b[1] = (int)((st >> 16) & 0xFFFF);
        w.b[2] = (int)((st >> 32) & 0xFFFF);
        uint64_t flags = st >> 48;
        const uint64_t off = S.koff ? S.koff[i] : (uint64_t)i * kk;
        const int ki = S.koff ? (int)S.kray[i] : kk;
        uint32_t *out = rbid + off;
        int cnt = 0;
        bool alive = !(flags & kDone);
        if (alive) {
            walk_init(w, g);
            if (flags & kStep) alive = walk_step(w, g);
        }
        flags &= ~(kStep | kBoxed);
        int lim[3];
        box_limits(w.r.sgn, P.occ.box + 8 * view, lim);
        int steps = 0;
        while (alive) {   // uniform across the group: every lane holds the same walk
            if (++steps > max_steps) {
                if (gl == 0) atomicOr(&ctr[C_BAD], 2u);
                alive = false;
                break;
            }
            const int *b = w.b;
            if (past_box(b, w.r.sgn, lim)) {
                alive = false;
                break;
            }
            const uint32_t sc =
                (uint32_t)(b[0] >> 4) + ns0 * ((uint32_t)(b[1] >> 4) + ns1 * (uint32_t)(b[2] >> 4));
            const uint32_t c =
                (uint32_t)(b[0] >> 2) + nc0 * ((uint32_t)(b[1] >> 2) + nc1 * (uint32_t)(b[2] >> 2));
            // both masks in flight at once (the coarse one is unused when the
            // super mask says the cell is empty)
            const unsigned long long smask = __ldg(sm + sc);
            const unsigned long long fmask = __ldg(fm + c);
            if (!mask_bit(smask, ((b[0] >> 2) & 3) + 4 * ((b[1] >> 2) & 3) + 16 * ((b[2] >> 2) & 3))) {
                alive = skip_level(w, g, smask ? 4 : 16, smask ? g.tc : P.occ.ts);
                continue;
            }

            // crossings inside this coarse cell per axis; the last one leaves it
            int na[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (w.r.sgn[a] > 0) na[a] = min(4 * (b[a] >> 2) + 4 - b[a], g.tb[a] - b[a]);
                else if (w.r.sgn[a] < 0) na[a] = b[a] - 4 * (b[a] >> 2) + 1;
                else na[a] = 0;
            }
            // time of the k-th crossing along axis a (exact numerator over |d_a|)
            auto cross = [&](int a, int k) -> Tq {
                const float X = w.r.sgn[a] > 0 ? (float)min(4 * (b[a] + k), g.dims[a] - 1) : (float)(4 * (b[a] - k + 1));
                const float n = __fsub_rn(X, w.r.e[a]);
                return Tq{w.r.sgn[a] > 0 ? n : -n, w.r.ad[a]};
            };
            Tq tex{0.f, 1.f};
            bool have = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (!na[a]) continue;
                const Tq t = cross(a, na[a]);
                if (!have || tcmp(t, tex) < 0) {
                    tex = t;
                    have = true;
                }
            }
            // this lane's crossing: crossings per axis up to its time (cle:
            // at or before, clt: strictly before); its axis's values are
            // selected, not indexed, so the walk stays in registers
            bool valid = false, rep = false, interior = false;
            int cle[3] = {0, 0, 0}, clt[3] = {0, 0, 0};
            const int na_e = ea == 0 ? na[0] : (ea == 1 ? na[1] : na[2]);
            if (elane && ek <= na_e) {
                const int sg = ea == 0 ? w.r.sgn[0] : (ea == 1 ? w.r.sgn[1] : w.r.sgn[2]);
                const int bq = ea == 0 ? b[0] : (ea == 1 ? b[1] : b[2]);
                const int dq = ea == 0 ? g.dims[0] : (ea == 1 ? g.dims[1] : g.dims[2]);
                const float eq = ea == 0 ? w.r.e[0] : (ea == 1 ? w.r.e[1] : w.r.e[2]);
                const float adq = ea == 0 ? w.r.ad[0] : (ea == 1 ? w.r.ad[1] : w.r.ad[2]);
                const float Xq = sg > 0 ? (float)min(4 * (bq + ek), dq - 1) : (float)(4 * (bq - ek + 1));
                const float nq = __fsub_rn(Xq, eq);
                const Tq tl{sg > 0 ? nq : -nq, adq};
                const int ce = tcmp(tl, tex);
                valid = ce <= 0;
                interior = ce < 0;
                if (valid) {
                    rep = true;
#pragma unroll
                    for (int a2 = 0; a2 < 3; ++a2) {
                        if (a2 == ea) {
                            cle[a2] = ek;
                            clt[a2] = ek - 1;
                            continue;
                        }
                        // crossing times grow with k2: count up to the first later one
                        for (int k2 = 1; k2 <= na[a2]; ++k2) {
                            const int cc = tcmp(cross(a2, k2), tl);
                            if (cc > 0) break;
                            ++cle[a2];
                            if (cc < 0) ++clt[a2];
                        }
                        if (a2 < ea && cle[a2] != clt[a2]) rep = false;   // a lower axis crosses at the same time
                    }
                }
            }
            const unsigned repm = __ballot_sync(full, valid && rep) >> gshift;
            const unsigned ltm = ((1u << clt[0]) - 1u) | (((1u << clt[1]) - 1u) << 4) | (((1u << clt[2]) - 1u) << 8);
            const int rank = __popc(repm & ltm);
            int nbk[3];
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) nbk[a2] = b[a2] + w.r.sgn[a2] * cle[a2];
            // positions in the cell: 0 = the current block, rank + 1 = the
            // block after an interior crossing
            bool vis = false;
            int pos = 0, bb[3] = {b[0], b[1], b[2]};
            if (gl == LPR - 1) {
                vis = mask_bit(fmask, (b[0] & 3) + 4 * (b[1] & 3) + 16 * (b[2] & 3));
            } else if (interior && rep) {
                pos = rank + 1;
                bb[0] = nbk[0];
                bb[1] = nbk[1];
                bb[2] = nbk[2];
                vis = mask_bit(fmask, (bb[0] & 3) + 4 * (bb[1] & 3) + 16 * (bb[2] & 3));
            }
            const unsigned vmask = __reduce_or_sync(full, vis ? (1u << pos) : 0u);
            const int need = ki - cnt;
            const int take = min(need, __popc(vmask));
            const int idx = vis ? __popc(vmask & ((1u << pos) - 1u)) : 32;
            if (idx < take) {
                const uint32_t blin = (uint32_t)bb[0] + nb0 * ((uint32_t)bb[1] + nb1 * (uint32_t)bb[2]);
                if (S.eray) S.eray[off + cnt + idx] = (uint32_t)i;
                out[cnt + idx] = blin;
                set_bit(vis_bits, blin);
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    int x = bb[0] + (o & 1), y = bb[1] + ((o >> 1) & 1), z = bb[2] + (o >> 2);
                    if (x < g.nb[0] && y < g.nb[1] && z < g.nb[2])
                        set_bit(act_bits, (uint32_t)x + nb0 * ((uint32_t)y + nb1 * (uint32_t)z));
                }
            }
            cnt += take;
            if (take == need) {   // k blocks taken: stop on the last one
                const int src = __ffs(__ballot_sync(full, idx == take - 1) >> gshift) - 1;
#pragma unroll
                for (int a2 = 0; a2 < 3; ++a2) w.b[a2] = __shfl_sync(full, bb[a2], src, LPR);
                flags |= kStep;
                break;
            }
            // on to the block after T_exit (the lowest axis crossing then)
            const int src = __ffs(__ballot_sync(full, valid && rep && !interior) >> gshift) - 1;
            bool inside = true;
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) {
                w.b[a2] = __shfl_sync(full, nbk[a2], src, LPR);
                if (w.b[a2] < 0 || w.b[a2] >= g.tb[a2]) inside = false;
            }
            if (!inside) {
                alive = false;
                break;
            }
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) set_axis(w, g, a2);
        }
        if (!alive) flags |= kDone;
        for (int j = cnt + gl; j < ki; j += LPR) out[j] = kNone;
        if (gl == 0) {
            state_out[ray] = pack_state(w.b, flags);
            tot_steps += (uint32_t)steps;
            max_seen = max(max_seen, (uint32_t)steps);
        }
    }
    if (gl == 0) {
        if (tot_steps) atomicAdd(&ctr[C_STEPS], tot_steps);
        if (max_seen) atomicMax(&ctr[C_MAXSTEPS], max_seen);
    }
}

// ----------------------------------------------------- segmented traversal
// A pass's walks are as long as its longest ray: one thread per ray leaves
// most lanes idle behind a few rays that cross the whole volume.  The
// segmented walk gives each live ray a group of SL lanes (a power of two,
// SL = seg_threads / nproc rounded down, at most 32).  The ray's remaining
// path is cut at block planes of its dominant axis (the axis of largest
// |d|; every block index along it changes monotonically): lane j owns the
// blocks whose index along that axis lies in the j-th of SL equal parts of
// the range from the current block to the block where the ray leaves the
// occupied box (the walk ends there).  Lane 0
// resumes the saved walk; lane j > 0 starts at the exact crossing time T_j
// of its first plane, in the block containing p(T_j+) (located with the
// exact predicates, the right-limit rule of the serial walk), unless the
// ray has left the volume by then.  Each lane then runs the serial walk
// (walk_step, skip_level, the brick masks) until its index leaves its part,
// the ray leaves the volume, or it holds k visible blocks.  Because the parts
// partition the path by a coordinate that only grows (or only shrinks), the
// concatenation of the lanes' visible blocks in lane order is the serial
// walk's sequence; the group keeps its first k (an exclusive scan of the
// counts) and marks only those.  Blocks are buffered in shared memory; a lane
// that found more than kSegBuf walks its part again, writing directly.
constexpr int kSegBuf = 32;
constexpr int kSegThreads = 128;

struct SegPart {
    int as;        // dominant axis
    int b0;        // index along it of the ray's current block
    int o0, o1;    // this lane's offsets [o0, o1) from b0 along the walk
};

// The dominant axis and this lane's part; false when the part is empty.
// The parts end at the block where the ray leaves the occupied box bx or
// the volume (the walk stops there), never before the current block.
__device__ __forceinline__ bool seg_part(const Walk &w, const VolGeom &g, const int *bx, int SL, int gl, SegPart &sp)
{
    int as = 0;
    float best = -1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (w.r.ad[a] > best) {
            best = w.r.ad[a];
            as = a;
        }
    sp.as = as;
    const int bq = as == 0 ? w.b[0] : (as == 1 ? w.b[1] : w.b[2]);
    const int sg = as == 0 ? w.r.sgn[0] : (as == 1 ? w.r.sgn[1] : w.r.sgn[2]);
    const int tbq = as == 0 ? g.tb[0] : (as == 1 ? g.tb[1] : g.tb[2]);
    sp.b0 = bq;
    // the ray leaves the box (or the volume) at T1, its first far-plane
    // crossing; the block holding p(T1+) bounds the walk along the dominant
    // axis (the walk's blocks before T1 lie between the current one and it)
    Tq t1{0.f, 1.f};
    bool have = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (w.r.sgn[a] == 0) continue;
        const float farp = w.r.sgn[a] > 0 ? fminf((float)(4 * (bx[4 + a] + 1)), (float)(g.dims[a] - 1))
                                           : fmaxf((float)(4 * bx[a]), 0.f);
        const Tq tf = plane_t(w.r, a, farp);
        if (!have || tcmp(tf, t1) < 0) {
            t1 = tf;
            have = true;
        }
    }
    const int loq = bx[as], hiq = bx[4 + as];
    const int span_box = max(1, sg > 0 ? min(tbq, hiq + 1) - bq : bq - max(loq, 0) + 1);
    const int bend = locate_block(w.r, as, t1, tbq);
    const int span = have ? max(1, min(span_box, (sg > 0 ? bend - bq : bq - bend) + 1)) : span_box;
    // rounded up, so that lane 0's part always holds the current block (only
    // lane 0 resumes the saved walk); later lanes may get empty parts
    sp.o0 = (int)(((int64_t)gl * span + SL - 1) / SL);
    sp.o1 = (int)(((int64_t)(gl + 1) * span + SL - 1) / SL);
    return sp.o0 < sp.o1;
}

__device__ __forceinline__ int seg_offset(const Walk &w, const SegPart &sp)
{
    const int bq = sp.as == 0 ? w.b[0] : (sp.as == 1 ? w.b[1] : w.b[2]);
    const int sg = sp.as == 0 ? w.r.sgn[0] : (sp.as == 1 ? w.r.sgn[1] : w.r.sgn[2]);
    return sg > 0 ? bq - sp.b0 : sp.b0 - bq;
}

// Place a lane's walk at the start of its part: lane 0 resumes the saved
// walk (stepping first when the saved block was already taken), lane j > 0
// starts in the block holding p(T_j+).  False when nothing is left to walk.
__device__ __forceinline__ bool seg_start(Walk &w, const VolGeom &g, const SegPart &sp, int gl, const int b_saved[3],
                                          bool step_first)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) w.b[a] = b_saved[a];
    if (gl == 0) {
        walk_init(w, g);
        return step_first ? walk_step(w, g) : true;
    }
    const int as = sp.as;
    const int sg = as == 0 ? w.r.sgn[0] : (as == 1 ? w.r.sgn[1] : w.r.sgn[2]);
    const int first = sg > 0 ? sp.b0 + sp.o0 : sp.b0 - sp.o0;        // first block index of the part
    const float X = (float)(sg > 0 ? 4 * first : 4 * (first + 1));   // the plane entering it
    const Tq T = plane_t(w.r, as, X);
    // the time the ray leaves the volume: its first far-plane crossing
    Tq tout{0.f, 1.f};
    bool have = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (w.r.sgn[a] == 0) continue;
        const Tq tf = plane_t(w.r, a, w.r.sgn[a] > 0 ? (float)(g.dims[a] - 1) : 0.f);
        if (!have || tcmp(tf, tout) < 0) {
            tout = tf;
            have = true;
        }
    }
    if (!have || tcmp(T, tout) >= 0) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) w.b[a] = a == as ? first : locate_block(w.r, a, T, g.tb[a]);
    walk_init(w, g);
    return true;
}

// One lane's walk over its part.  Emit mode 0 buffers up to kSegBuf blocks
// (and the step count at each) in shared memory; mode 1 writes blocks
// q < n_write directly to out[q] and marks them.  Returns the visible blocks
// found (at most cap); *end_steps the steps taken, *exited whether the walk
// left the volume, *last the last block written in mode 1.
struct SegOut {
    uint32_t *blk;      // shared: [kSegBuf][kSegThreads], this thread's column
    uint16_t *stp;
    uint32_t *out;      // mode 1
    uint32_t *eray;     // mode 1, per-ray speculation (may be null)
    uint32_t ray_pos;
    uint32_t *vis_bits, *act_bits;
};

template <int MODE>
__device__ __forceinline__ int seg_walk(Walk &w, const Geo &P, const SegPart &sp, int view, int cap, int n_write, const SegOut &o,
                        int max_steps, uint32_t *ctr, int *end_steps, bool *exited, uint32_t *last)
{
    const VolGeom &g = P.g;
    const unsigned long long *fm = P.occ.fmask + view * P.fstride, *sm = P.occ.smask + view * P.sstride;
    const uint32_t nb0 = g.nb[0], nb1 = g.nb[1], nc0 = g.nc[0], nc1 = g.nc[1];
    const uint32_t ns0 = P.occ.ns[0], ns1 = P.occ.ns[1];
    int lim[3];
    box_limits(w.r.sgn, P.occ.box + 8 * view, lim);
    int cnt = 0, steps = 0;
    bool alive = true;
    uint32_t cur_s = 0xFFFFFFFFu, cur_c = 0xFFFFFFFFu;
    unsigned long long smask = 0ull, fmask = 0ull;
    while (alive) {
        if (seg_offset(w, sp) >= sp.o1) break;   // the next lane's part
        if (++steps > max_steps) {
            atomicOr(&ctr[C_BAD], 2u);
            alive = false;
            break;
        }
        const int *b = w.b;
        if (past_box(b, w.r.sgn, lim)) {
            alive = false;
            break;
        }
        const uint32_t sc = (uint32_t)(b[0] >> 4) + ns0 * ((uint32_t)(b[1] >> 4) + ns1 * (uint32_t)(b[2] >> 4));
        if (sc != cur_s) {
            smask = __ldg(sm + sc);
            cur_s = sc;
        }
        if (!mask_bit(smask, ((b[0] >> 2) & 3) + 4 * ((b[1] >> 2) & 3) + 16 * ((b[2] >> 2) & 3))) {
            alive = skip_level(w, g, smask ? 4 : 16, smask ? g.tc : P.occ.ts);
            continue;
        }
        const uint32_t c = (uint32_t)(b[0] >> 2) + nc0 * ((uint32_t)(b[1] >> 2) + nc1 * (uint32_t)(b[2] >> 2));
        if (c != cur_c) {
            fmask = __ldg(fm + c);
            cur_c = c;
        }
        if (mask_bit(fmask, (b[0] & 3) + 4 * (b[1] & 3) + 16 * (b[2] & 3))) {
            const uint32_t blin = (uint32_t)b[0] + nb0 * ((uint32_t)b[1] + nb1 * (uint32_t)b[2]);
            if (MODE == 0) {
                if (cnt < kSegBuf) {
                    o.blk[cnt * kSegThreads] = blin;
                    o.stp[cnt * kSegThreads] = (uint16_t)min(steps, 65535);
                }
            } else if (cnt < n_write) {
                o.out[cnt] = blin;
                if (o.eray) o.eray[cnt] = o.ray_pos;
                set_bit(o.vis_bits, blin);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    int x = b[0] + (q & 1), y = b[1] + ((q >> 1) & 1), z = b[2] + (q >> 2);
                    if (x < g.nb[0] && y < g.nb[1] && z < g.nb[2])
                        set_bit(o.act_bits, (uint32_t)x + nb0 * ((uint32_t)y + nb1 * (uint32_t)z));
                }
                *last = blin;
            }
            if (++cnt == cap) break;
            if (MODE == 1 && cnt >= n_write) break;
        }
        alive = walk_step(w, g);
    }
    *end_steps = steps;
    *exited = !alive;
    return cnt;
}

__global__ void __launch_bounds__(kSegThreads, 6) traverse_seg_kernel(Geo P, const uint32_t *__restrict__ live0,
                                                                   const uint32_t *__restrict__ live1,
                                                                   const PassState *__restrict__ ps,
                                                                   const uint64_t *__restrict__ state_in,
                                                                   uint64_t *__restrict__ state_out,
                                                                   uint32_t *__restrict__ rbid,
                                                                   uint32_t *vis_bits, uint32_t *act_bits,
                                                                   uint32_t *ctr, Spec S)
{
    __shared__ uint32_t s_blk[kSegBuf * kSegThreads];
    __shared__ uint16_t s_stp[kSegBuf * kSegThreads];
    const int SL = seg_lanes(ps);
    if (SL < 2) return;
    const VolGeom &g = P.g;
    const uint32_t nproc = ps->nproc;
    const int kk = (int)ps->kk;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    const int max_steps = 2 * (g.tb[0] + g.tb[1] + g.tb[2]) + 8;
    const int lg = 31 - __clz(SL);
    const int lane = threadIdx.x & 31;
    const int gl = lane & (SL - 1);
    const unsigned gmask = SL == 32 ? 0xFFFFFFFFu : (((1u << SL) - 1u) << (lane & ~(SL - 1)));
    const uint32_t nb0 = g.nb[0], nb1 = g.nb[1];
    SegOut o{s_blk + threadIdx.x, s_stp + threadIdx.x, nullptr, nullptr, 0u, vis_bits, act_bits};
    uint32_t tot_steps = 0, max_seen = 0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> lg; i < nproc;
         i += ((int64_t)gridDim.x * blockDim.x) >> lg) {
        const uint32_t ray = live[i];
        Walk w;
        int view, px, py;
        ray_pixel(P, ray, view, px, py);
        {
            const Cam &cam = P.views[view].cam;
            make_ray(w.r, cam.eye, cam.p00, cam.du, cam.dv, px, py);
        }
        const uint64_t st = state_in[ray];
        const int b_saved[3] = {(int)(st & 0xFFFF), (int)((st >> 16) & 0xFFFF), (int)((st >> 32) & 0xFFFF)};
        const uint64_t flags = st >> 48;
        const uint64_t off = S.koff ? S.koff[i] : (uint64_t)i * kk;
        const int ki = S.koff ? (int)S.kray[i] : kk;
        uint32_t *out = rbid + off;

        // 1. this lane's part, walked with the blocks buffered
        int cnt = 0, steps = 0;
        bool exited = false;
        SegPart sp;
        bool active = false;
        if (!(flags & kDone)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) w.b[a] = b_saved[a];
            if (seg_part(w, g, P.occ.box + 8 * view, SL, gl, sp)) active = seg_start(w, g, sp, gl, b_saved, (flags & kStep) != 0);
            else if (gl == 0) active = false;
            if (gl == 0 && !active) exited = true;   // lane 0's step left the volume
        } else {
            exited = true;
        }
        uint32_t dummy = 0;
        if (active) cnt = seg_walk<0>(w, P, sp, view, ki, 0, o, max_steps, ctr, &steps, &exited, &dummy);
        // 2. the group's order: exclusive scan of the counts
        int incl = cnt;
        for (int d = 1; d < SL; d <<= 1) {
            const int y = __shfl_up_sync(gmask, incl, d, SL);
            if (gl >= d) incl += y;
        }
        const int pre = incl - cnt;
        const int total = __shfl_sync(gmask, incl, SL - 1, SL);
        const int n_write = max(0, min(cnt, ki - pre));
        // 3. the first k blocks of the ray: written and marked
        uint32_t last = kNone;
        if (n_write > 0 && n_write <= kSegBuf) {
            for (int q = 0; q < n_write; ++q) {
                const uint32_t blin = s_blk[q * kSegThreads + threadIdx.x];
                out[pre + q] = blin;
                if (S.eray) S.eray[off + pre + q] = (uint32_t)i;
                set_bit(vis_bits, blin);
                const int bx = (int)(blin % nb0), by = (int)((blin / nb0) % nb1), bz = (int)(blin / (nb0 * nb1));
#pragma unroll
                for (int q2 = 0; q2 < 8; ++q2) {
                    int x = bx + (q2 & 1), y = by + ((q2 >> 1) & 1), z = bz + (q2 >> 2);
                    if (x < g.nb[0] && y < g.nb[1] && z < g.nb[2])
                        set_bit(act_bits, (uint32_t)x + nb0 * ((uint32_t)y + nb1 * (uint32_t)z));
                }
                last = blin;
            }
        } else if (n_write > 0) {   // more than the buffer holds: walk the part again, writing
            SegOut o2 = o;
            o2.out = out + pre;
            o2.eray = S.eray ? S.eray + off + pre : nullptr;
            o2.ray_pos = (uint32_t)i;
            int s2 = 0;
            bool e2 = false;
            seg_start(w, g, sp, gl, b_saved, (flags & kStep) != 0);
            seg_walk<1>(w, P, sp, view, ki, n_write, o2, max_steps, ctr, &s2, &e2, &last);
        }
        for (int j = min(total, ki) + gl; j < ki; j += SL) out[j] = kNone;
        // 4. state: after the k-th block, or done (every part walked, fewer
        // than k found: the ray leaves the volume)
        const bool holds_kth = pre < ki && pre + cnt >= ki;
        if (total >= ki) {
            if (holds_kth) {
                const int bq[3] = {(int)(last % nb0), (int)((last / nb0) % nb1), (int)(last / (nb0 * nb1))};
                state_out[ray] = pack_state(bq, kStep);
            }
        } else if (gl == 0) {
            state_out[ray] = pack_state(b_saved, kDone);
        }
        // useful steps: whole parts before the k-th block, up to it in its part
        int useful = 0;
        if (pre < ki) {
            if (holds_kth) {
                const int q = ki - 1 - pre;
                useful = q < kSegBuf ? (int)s_stp[q * kSegThreads + threadIdx.x] : steps;
            } else {
                useful = steps;
            }
        }
        tot_steps += (uint32_t)useful;
        max_seen = max(max_seen, (uint32_t)useful);
        (void)exited;
    }
    warp_add(&ctr[C_STEPS], tot_steps);
    {
        unsigned m = __activemask();
        uint32_t mx = __reduce_max_sync(m, max_seen);
        if ((threadIdx.x & 31) == (unsigned)(__ffs(m) - 1) && mx) atomicMax(&ctr[C_MAXSTEPS], mx);
    }
}

// --------------------------------------------------------------- grouping
struct BitsEmit {
    const uint32_t *bits;
    uint32_t *wpre;  // optional: the prefix of each word that holds a set bit
    uint32_t *list;
    uint32_t *zero;  // optional: zero this array at each emitted position
    __device__ void operator()(int64_t w, uint32_t pre, uint32_t c) const
    {
        if (!c) return;   // empty words: no prefix is ever asked for them
        if (wpre) wpre[w] = pre;
        uint32_t x = bits[w];
        while (x) {
            int k = __ffs(x) - 1;
            x &= x - 1;
            list[pre] = (uint32_t)(w * 32 + k);
            if (zero) zero[pre] = 0u;
            ++pre;
        }
    }
};


__device__ __forceinline__ uint32_t vis_rank(const uint32_t *bits, const uint32_t *wpre, uint32_t b)
{
    uint32_t w = b >> 5;
    return wpre[w] + __popc(bits[w] & ((1u << (b & 31)) - 1u));
}

// Compaction of a block bitmap (one bit per block: millions of words, few
// set bits).  The single-pass look-back is bound there by how far each
// tile's prefix travels: the CTAs of the first wave run at once, and the
// last of them adds hundreds of predecessors' aggregates, 32 per round.
// Two kernels instead: bits_reduce_kernel counts each tile's bits;
// bits_emit_kernel adds the counts of the tiles before its own (a few
// thousand at most, read from L2), scans its words and emits their bits in
// order.  Same outputs as a compact_kernel over the words' popcounts.
constexpr int kBitsThreads = 256, kBitsWords = 8;   // a multiple of 4
constexpr int64_t kBitsTile = (int64_t)kBitsThreads * kBitsWords;   // words per tile

inline int64_t bits_tiles(int64_t nwords) { return std::max<int64_t>(1, (nwords + kBitsTile - 1) / kBitsTile); }

// this thread's kBitsWords words (16-byte loads when all lie below n)
__device__ __forceinline__ void load_words(const uint32_t *bits, int64_t first, int64_t n, uint32_t w[kBitsWords])
{
    if (first + kBitsWords <= n) {
#pragma unroll
        for (int q = 0; q < kBitsWords / 4; ++q) {
            const uint4 a = *reinterpret_cast<const uint4 *>(bits + first + 4 * q);
            w[4 * q] = a.x, w[4 * q + 1] = a.y, w[4 * q + 2] = a.z, w[4 * q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kBitsWords; ++j) w[j] = first + j < n ? bits[first + j] : 0u;
    }
}

__global__ void __launch_bounds__(kBitsThreads) bits_reduce_kernel(const uint32_t *__restrict__ bits, int64_t n,
                                                                   uint32_t *__restrict__ tile_sum)
{
    __shared__ uint32_t s_w[kBitsThreads / 32];
    uint32_t w[kBitsWords];
    load_words(bits, (int64_t)blockIdx.x * kBitsTile + (int64_t)threadIdx.x * kBitsWords, n, w);
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kBitsWords; ++j) c += __popc(w[j]);
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
#pragma unroll
        for (int i = 0; i < kBitsThreads / 32; ++i) t += s_w[i];
        tile_sum[blockIdx.x] = t;
    }
}

// total (and *over = total > over_limit, when over is given) from the last
// tile's last thread; with clear, each word is zeroed once its bits are
// emitted (the bitmap is then all zero, as a memset would leave it)
template <class EmitF>
__global__ void __launch_bounds__(kBitsThreads) bits_emit_kernel(uint32_t *__restrict__ bits, int64_t n,
                                                                 const uint32_t *__restrict__ tile_sum, EmitF emit,
                                                                 uint32_t *total, uint32_t *over, uint32_t over_limit,
                                                                 bool clear)
{
    __shared__ uint32_t s_w[kBitsThreads / 32];
    __shared__ uint32_t s_pre;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // the tile's prefix: the bits of the tiles before it
    uint32_t acc = 0;
    for (int64_t t = threadIdx.x; t < (int64_t)blockIdx.x; t += kBitsThreads) acc += tile_sum[t];
    acc = __reduce_add_sync(0xFFFFFFFFu, acc);
    if (lane == 0) s_w[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
#pragma unroll
        for (int i = 0; i < kBitsThreads / 32; ++i) t += s_w[i];
        s_pre = t;
    }
    __syncthreads();
    // this thread's words and their exclusive prefix within the tile
    const int64_t first = (int64_t)blockIdx.x * kBitsTile + (int64_t)threadIdx.x * kBitsWords;
    uint32_t w[kBitsWords], c[kBitsWords], local = 0;
    load_words(bits, first, n, w);
#pragma unroll
    for (int j = 0; j < kBitsWords; ++j) {
        c[j] = __popc(w[j]);
        local += c[j];
    }
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t v = lane < kBitsThreads / 32 ? s_w[lane] : 0u;
        uint32_t vi = v;
#pragma unroll
        for (int o = 1; o < kBitsThreads / 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, vi, o);
            if (lane >= o) vi += y;
        }
        if (lane < kBitsThreads / 32) s_w[lane] = vi - v;   // exclusive warp offsets
    }
    __syncthreads();
    uint32_t run = s_pre + s_w[wid] + incl - local;
#pragma unroll
    for (int j = 0; j < kBitsWords; ++j) {
        if (first + j < n) emit(first + j, run, c[j]);
        run += c[j];
    }
    if (clear) {
#pragma unroll
        for (int j = 0; j < kBitsWords; ++j)
            if (w[j]) bits[first + j] = 0u;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kBitsThreads - 1) {
        if (total) *total = run;
        if (over) *over = run > over_limit ? 1u : 0u;
    }
}

__global__ void count_entries_kernel(const PassState *ps, const uint32_t *__restrict__ rbid, const uint32_t *vis_bits,
                                     const uint32_t *vis_wpre, uint32_t *nbrays, uint32_t *erank,
                                     const uint32_t *ctr, Spec S)
{
    if (ctr[C_OVERFLOW]) return;
    const int64_t n = S.koff ? (int64_t)ctr[C_KTOT] : (int64_t)ps->nproc * ps->kk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = rbid[e];
        if (b == kNone) continue;
        erank[e] = atomicAdd(&nbrays[vis_rank(vis_bits, vis_wpre, b)], 1u);
    }
}

struct ArrayCount {
    const uint32_t *a;
    const uint32_t *skip;
    __device__ bool enabled() const { return !skip || !*skip; }
    __device__ uint32_t operator()(int64_t i) const { return a[i]; }
};

struct ArrayEmit {
    uint32_t *out;
    __device__ void operator()(int64_t i, uint32_t pre, uint32_t) const { out[i] = pre; }
};

__global__ void scatter_entries_kernel(const PassState *ps, const uint32_t *__restrict__ rbid, const uint32_t *vis_bits,
                                       const uint32_t *vis_wpre, const uint32_t *obrays,
                                       const uint32_t *erank, uint32_t *E, const uint32_t *ctr, Spec S)
{
    if (ctr[C_OVERFLOW]) return;
    const int64_t n = S.koff ? (int64_t)ctr[C_KTOT] : (int64_t)ps->nproc * ps->kk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = rbid[e];
        if (b == kNone) continue;
        E[obrays[vis_rank(vis_bits, vis_wpre, b)] + erank[e]] = (uint32_t)e;
    }
}

// ------------------------------------------------------------------ cache
// The count only reads (1 for a miss), so a thread's lookups are issued
// together; the emit marks the hits' slots touched (a byte store, which the
// compiler must assume may alias the tables, would otherwise order every
// later lookup after it).
struct LookupCount {
    const uint32_t *iact;
    const uint32_t *blk_slot;
    const uint32_t *skip;
    __device__ bool enabled() const { return !*skip; }
    __device__ uint32_t operator()(int64_t i) const { return __ldg(blk_slot + __ldg(iact + i)) == kNone ? 1u : 0u; }
};

// misses listed in order; hits' slots marked touched
struct LookupEmit {
    const uint32_t *iact;
    const uint32_t *blk_slot;
    uint8_t *touched;
    uint32_t *miss;
    __device__ void operator()(int64_t i, uint32_t pre, uint32_t c) const
    {
        const uint32_t b = __ldg(iact + i);
        if (c) miss[pre] = b;
        else touched[__ldg(blk_slot + b)] = 1;
    }
};


// the LRU list in use and the one being built, chosen by the pass parity
struct LruPair {
    uint32_t *l0, *l1;
    const PassState *ps;
    __device__ uint32_t *cur() const { return (ps->parity & 2) ? l1 : l0; }
    __device__ uint32_t *next() const { return (ps->parity & 2) ? l0 : l1; }
};

// misses served from never-used slots; the rest come from the used list
__device__ __forceinline__ uint32_t fresh_taken(const PassState *ps, const uint32_t *ctr, uint32_t n_slots)
{
    return min(ctr[C_NMISS], n_slots - ps->fresh_lo);
}

// Untouched used slots in LRU order, before the assignment: the first ones
// become victims.  Runs only when the never-used slots do not cover the
// misses (otherwise no victim is taken and the scan is skipped).
struct VictimCount {
    LruPair lru;
    const uint8_t *touched;
    const uint32_t *ctr;
    uint32_t n_slots;
    __device__ bool enabled() const
    {
        return !ctr[C_OVERFLOW] && ctr[C_NMISS] > fresh_taken(lru.ps, ctr, n_slots);
    }
    __device__ uint32_t operator()(int64_t i) const { return touched[lru.cur()[i]] ? 0u : 1u; }
};

struct VictimEmit {
    LruPair lru;
    const uint32_t *ctr;
    uint32_t *victim;
    uint32_t n_slots;
    __device__ void operator()(int64_t i, uint32_t pre, uint32_t c) const
    {
        if (!c) return;
        const uint32_t nf = fresh_taken(lru.ps, ctr, n_slots);
        if (pre < ctr[C_NMISS] - nf) victim[nf + pre] = lru.cur()[i];
    }
};

// After the assignment (which marks the victims and the fresh slots it
// hands out): the used slots still untouched, in LRU order, start the next
// pass's list (the victims were the first untouched ones before it, so the
// rest keep their order).  Off the decode's path.
struct KeepCount {
    LruPair lru;
    const uint8_t *touched;
    const uint32_t *skip;
    __device__ bool enabled() const { return !*skip; }
    __device__ uint32_t operator()(int64_t i) const { return touched[lru.cur()[i]] ? 0u : 1u; }
};

struct KeepEmit {
    LruPair lru;
    __device__ void operator()(int64_t i, uint32_t pre, uint32_t c) const
    {
        if (c) lru.next()[pre] = lru.cur()[i];
    }
};

// The cache assignment of the pass's misses, done by the decoder as it reads
// each miss (decode_sorted_kernel's slot functor), so that it takes no launch
// of its own on the way to the decode: miss i takes never-used slot
// fresh_lo + i while those last, else victim[i] (the least recently used
// untouched slot); the slot's previous block loses its mapping; block and
// slot map to each other; the slot is marked touched.
struct AssignSlot {
    const uint32_t *victim;
    uint32_t *blk_slot, *slot_blk;
    uint8_t *touched;
    uint32_t *ctr;
    PassState *ps;
    uint32_t n_slots;
    __device__ void begin() const
    {
        const uint32_t nf = fresh_taken(ps, ctr, n_slots);
        ps->fresh_hi = ps->fresh_lo + nf;
        ctr[C_NEEDUSED] = ctr[C_NMISS] - nf;
    }
    __device__ uint32_t operator()(int64_t i, uint32_t b) const
    {
        const uint32_t nf = fresh_taken(ps, ctr, n_slots);
        const uint32_t s = i < nf ? ps->fresh_lo + (uint32_t)i : victim[i];
        const uint32_t old = slot_blk[s];
        uint32_t ev = 0;
        if (old != kNone) {
            blk_slot[old] = kNone;
            ev = 1;
        }
        blk_slot[b] = s;
        slot_blk[s] = b;
        touched[s] = 1;
        warp_add(&ctr[C_EVICT], ev);
        return s;
    }
};

struct TouchedCount {
    const uint8_t *touched;
    const uint32_t *skip;
    __device__ bool enabled() const { return !*skip; }
    __device__ uint32_t operator()(int64_t s) const { return touched[s] ? 1u : 0u; }
};

// touched slots (hits and victims), all below fresh_hi, appended in slot order
struct TouchedEmit {
    uint8_t *touched;
    const uint32_t *ctr;
    LruPair lru;
    __device__ void operator()(int64_t s, uint32_t pre, uint32_t c) const
    {
        if (!c) return;
        lru.next()[ctr[C_NUNTOUCHED] + pre] = (uint32_t)s;
        touched[s] = 0;
    }
};

__global__ void lru_init_kernel(uint32_t *lru, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lru[i] = (uint32_t)i;
}

// -------------------------------------------------------------- intersect
struct RT {
    Geo P;
    const float *cache;
    const uint32_t *blk_slot;
};

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

__device__ __forceinline__ float tri8(const float v[8], float x, float y, float z)
{
    float c00 = lerpf(v[0], v[1], x), c10 = lerpf(v[2], v[3], x);
    float c01 = lerpf(v[4], v[5], x), c11 = lerpf(v[6], v[7], x);
    return lerpf(lerpf(c00, c10, y), lerpf(c01, c11, y), z);
}

struct CellF {
    float v[8];
    float iso, u[3], d[3];
    __device__ float operator()(float s) const
    {
        return tri8(v, fmaf(s, d[0], u[0]), fmaf(s, d[1], u[1]), fmaf(s, d[2], u[2])) - iso;
    }
};

// power-basis coefficients of f along the segment: f(s) - f(0) = c1 s + c2 s^2 + c3 s^3.
// The trilinear form is multiplied out one axis at a time: the four x-edge
// interpolants are linear in s, the two y-interpolants of them quadratic, the
// z-interpolant of those cubic.
__device__ __forceinline__ void cubic_coeffs(const CellF &f, float &c1, float &c2, float &c3)
{
    float a[4], b[4];   // x-edge j + 2l: a + b s
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float v0 = f.v[2 * e], dv = f.v[2 * e + 1] - v0;
        a[e] = fmaf(dv, f.u[0], v0);
        b[e] = dv * f.d[0];
    }
    float p[2][3];   // y-interpolant at z level l: p0 + p1 s + p2 s^2
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float da = a[2 * l + 1] - a[2 * l], db = b[2 * l + 1] - b[2 * l];
        p[l][0] = fmaf(da, f.u[1], a[2 * l]);
        p[l][1] = fmaf(da, f.d[1], fmaf(db, f.u[1], b[2 * l]));
        p[l][2] = db * f.d[1];
    }
    const float r0 = p[1][0] - p[0][0], r1 = p[1][1] - p[0][1], r2 = p[1][2] - p[0][2];
    c1 = fmaf(r0, f.d[2], fmaf(r1, f.u[2], p[0][1]));
    c2 = fmaf(r1, f.d[2], fmaf(r2, f.u[2], p[0][2]));
    c3 = r2 * f.d[2];
}

// roots of f'(s) = 3 c3 s^2 + 2 c2 s + c1 inside (0, L), ascending, in e0 and
// e1 (returns how many); the coefficients are re-derived in double precision
// when the discriminant is ill-conditioned
__device__ __forceinline__ int deriv_roots(const CellF &f, float c1, float c2, float c3, float L, float &e0,
                                           float &e1)
{
    float a = 3.f * c3, b = 2.f * c2, c = c1;
    float disc = b * b - 4.f * a * c;
    float r0 = 0.f, r1 = 0.f;
    int n = 0;
    if (fabsf(disc) < 1e-5f * (b * b + fabsf(4.f * a * c))) {
        double C1 = 0.0, C2 = 0.0, C3 = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool i = k & 1, j = (k >> 1) & 1, l = k >> 2;
            double ax = i ? f.u[0] : 1.0 - f.u[0], bx = i ? f.d[0] : -(double)f.d[0];
            double ay = j ? f.u[1] : 1.0 - f.u[1], by = j ? f.d[1] : -(double)f.d[1];
            double az = l ? f.u[2] : 1.0 - f.u[2], bz = l ? f.d[2] : -(double)f.d[2];
            C1 += f.v[k] * (bx * ay * az + ax * by * az + ax * ay * bz);
            C2 += f.v[k] * (bx * by * az + bx * ay * bz + ax * by * bz);
            C3 += f.v[k] * (bx * by * bz);
        }
        double A = 3.0 * C3, B = 2.0 * C2, CC = C1;
        if (A == 0.0) {
            if (B != 0.0) {
                r0 = (float)(-CC / B);
                n = 1;
            }
        } else {
            double D = B * B - 4.0 * A * CC;
            if (D >= 0.0) {
                double q = -0.5 * (B + (B >= 0.0 ? sqrt(D) : -sqrt(D)));
                if (q != 0.0) {
                    r0 = (float)(q / A);
                    r1 = (float)(CC / q);
                    n = 2;
                } else {
                    n = 1;
                }
            }
        }
    } else if (a == 0.f) {
        if (b != 0.f) {
            r0 = -c / b;
            n = 1;
        }
    } else if (disc > 0.f) {
        float q = -0.5f * (b + copysignf(sqrtf(disc), b));
        if (q != 0.f) {
            r0 = q / a;
            r1 = c / q;
            n = 2;
        }
    }
    // keep those inside (0, L), ascending
    const bool in0 = n >= 1 && r0 > 0.f && r0 < L, in1 = n >= 2 && r1 > 0.f && r1 < L;
    if (in0 && in1) {
        e0 = fminf(r0, r1);
        e1 = fmaxf(r0, r1);
        return 2;
    }
    if (in0 || in1) {
        e0 = in0 ? r0 : r1;
        return 1;
    }
    return 0;
}

// a root of f in [a, b] where f(a), f(b) differ in sign: Newton steps on the
// trilinear f with the cubic's derivative, kept inside the shrinking bracket
// (bisection when a step leaves it), until the step is below 1e-6 (1 + s) --
// three orders of magnitude inside the depth tolerance
__device__ __forceinline__ float refine_root(const CellF &f, float c1, float c2, float c3, float a, float b,
                                             float fa, float fb)
{
    float s = a - fa * (b - a) / (fb - fa);   // secant start
    if (!(s > a && s < b)) s = 0.5f * (a + b);
    const bool neg_a = fa < 0.f;
    for (int it = 0; it < 40; ++it) {
        const float fs = f(s);
        if (fs == 0.f) return s;
        if ((fs < 0.f) == neg_a) a = s;
        else b = s;
        const float d = fmaf(fmaf(3.f * c3, s, 2.f * c2), s, c1);
        float sn = s - fs / d;
        if (!(sn > a && sn < b)) sn = 0.5f * (a + b);
        const float tol = 1e-6f * (1.f + fabsf(sn));
        if (fabsf(sn - s) <= tol || b - a <= tol) return sn;
        s = sn;
    }
    return 0.5f * (a + b);
}

// first root of f on [0, L]: monotone pieces split at the roots of f', the
// first piece that starts on a zero or changes sign, refined by refine_root
__device__ __forceinline__ bool first_root(const CellF &f, float L, float &s_hit)
{
    float c1, c2, c3;
    cubic_coeffs(f, c1, c2, c3);
    float e0 = L, e1 = L;
    const int ne = deriv_roots(f, c1, c2, c3, L, e0, e1);
    float fa = f(0.f);
    if (fa == 0.f) {
        s_hit = 0.f;
        return true;
    }
    float sa = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i > ne) break;
        const float sb = i == ne ? L : (i == 0 ? e0 : e1);
        const float fb = f(sb);
        if (fb == 0.f) {
            s_hit = sb;
            return true;
        }
        if ((fb < 0.f) != (fa < 0.f)) {
            s_hit = refine_root(f, c1, c2, c3, sa, sb, fa, fb);
            return true;
        }
        sa = sb;
        fa = fb;
    }
    return false;
}

// Intersect the ray with the isosurface inside block (bx,by,bz).  On a hit,
// returns the 44 low bits of the resolve key: depth bits, local cell, grey.
// The block's dual grid (its 4^3 voxels and the +x/+y/+z neighbours' face,
// edge and corner voxels, 5^3 values) as the intersection reads it: local
// corner (lx, ly, lz), each in 0..4, taken 8 at a time, a cell's corners.
// GlobalCorners reads each corner from the cache slot holding it (L1-cached
// loads); SharedCorners from a copy of the 5^3 values staged in shared memory.
struct GlobalCorners {
    const float *cache;
    uint32_t slots[8];   // own, +x, +y, +xy, +z, +xz, +yz, +xyz
    // the 8 corners of cell c (each 0..3), v[k] = corner (c + (k&1, k>>1&1,
    // k>>2)): a corner lies in the +a neighbour exactly when its offset along
    // a is 1 and c[a] == 3, so one cell's 8 slots follow from three flags
    __device__ __forceinline__ void load8(const int c[3], float v[8]) const
    {
        const bool xs = c[0] == 3, ys = c[1] == 3, zs = c[2] == 3;
        const uint32_t s000 = slots[0];
        const uint32_t s100 = xs ? slots[1] : s000;
        const uint32_t s010 = ys ? slots[2] : s000;
        const uint32_t s110 = ys ? (xs ? slots[3] : slots[2]) : s100;
        const uint32_t s001 = zs ? slots[4] : s000;
        const uint32_t s101 = zs ? (xs ? slots[5] : slots[4]) : s100;
        const uint32_t s011 = zs ? (ys ? slots[6] : slots[4]) : s010;
        const uint32_t s111 = zs ? (ys ? (xs ? slots[7] : slots[6]) : (xs ? slots[5] : slots[4])) : s110;
        const int x0 = c[0], x1 = (c[0] + 1) & 3, y0 = 4 * c[1], y1 = 4 * ((c[1] + 1) & 3), z0 = 16 * c[2],
                  z1 = 16 * ((c[2] + 1) & 3);
        v[0] = __ldg(cache + (uint64_t)s000 * 64 + (x0 + y0 + z0));
        v[1] = __ldg(cache + (uint64_t)s100 * 64 + (x1 + y0 + z0));
        v[2] = __ldg(cache + (uint64_t)s010 * 64 + (x0 + y1 + z0));
        v[3] = __ldg(cache + (uint64_t)s110 * 64 + (x1 + y1 + z0));
        v[4] = __ldg(cache + (uint64_t)s001 * 64 + (x0 + y0 + z1));
        v[5] = __ldg(cache + (uint64_t)s101 * 64 + (x1 + y0 + z1));
        v[6] = __ldg(cache + (uint64_t)s011 * 64 + (x0 + y1 + z1));
        v[7] = __ldg(cache + (uint64_t)s111 * 64 + (x1 + y1 + z1));
    }
};

struct SharedCorners {
    const float *v;   // 125 values, x fastest
    __device__ __forceinline__ void load8(const int c[3], float out[8]) const
    {
        const float *p = v + c[0] + 5 * c[1] + 25 * c[2];
        out[0] = p[0];
        out[1] = p[1];
        out[2] = p[5];
        out[3] = p[6];
        out[4] = p[25];
        out[5] = p[26];
        out[6] = p[30];
        out[7] = p[31];
    }
};

// cells per axis of block (bx, by, bz) that exist (1..4)
__device__ __forceinline__ void block_extent(const VolGeom &g, int bx, int by, int bz, int ext[3])
{
    ext[0] = min(4, g.dims[0] - 1 - 4 * bx);
    ext[1] = min(4, g.dims[1] - 1 - 4 * by);
    ext[2] = min(4, g.dims[2] - 1 - 4 * bz);
}

// the cache slots of a block and of the +x/+y/+z neighbours its cells reach
__device__ __forceinline__ void neighbour_slots(const RT &R, int bx, int by, int bz, const int ext[3],
                                                uint32_t slots[8])
{
    const VolGeom &g = R.P.g;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int x = bx + (k & 1), y = by + ((k >> 1) & 1), z = bz + (k >> 2);
        bool need = (!(k & 1) || ext[0] == 4) && (!(k & 2) || ext[1] == 4) && (!(k & 4) || ext[2] == 4);
        slots[k] = (need && x < g.nb[0] && y < g.nb[1] && z < g.nb[2])
                       ? R.blk_slot[x + (int64_t)g.nb[0] * (y + (int64_t)g.nb[1] * z)]
                       : 0u;
    }
}

template <class Corners>
__device__ bool intersect_block(const RT &R, const Ray &r, float isov, int bx, int by, int bz, const Corners &corner,
                                uint64_t &payload)
{
    const VolGeom &g = R.P.g;
    const float iso = isov;
    const int bq[3] = {bx, by, bz};
    float o[3];
    int ext[3];
    block_extent(g, bx, by, bz, ext);
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = __fsub_rn(r.e[a], (float)(4 * bq[a]));   // exact
    // entry into the block: the latest near-plane crossing (exact; ties go to
    // the higher axis, which is crossed last)
    int ain = -1;
    Tq tin{0.f, 1.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (r.sgn[a] == 0) continue;
        float Pn = r.sgn[a] > 0 ? 0.f : (float)ext[a];
        Tq t{r.sgn[a] > 0 ? __fsub_rn(Pn, o[a]) : __fsub_rn(o[a], Pn), r.ad[a]};
        if (ain < 0 || tcmp(t, tin) >= 0) {
            tin = t;
            ain = a;
        }
    }
    float q[3];
    float th = 0.f, tl = 0.f;  // t at the block entry as a float pair
    if (ain < 0 || tin.n <= 0.f) {
        q[0] = o[0];
        q[1] = o[1];
        q[2] = o[2];
    } else {
        const float ad = r.ad[ain];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a == ain) {
                q[a] = r.sgn[a] > 0 ? 0.f : (float)ext[a];
                continue;
            }
            // q_a = o_a + t_in d_a = (o_a |d_in| + n_in d_a) / |d_in|, numerator
            // formed with error-free products so that the cancellation is exact
            float p1, e1, p2, e2, s, es;
            two_prod(o[a], ad, p1, e1);
            two_prod(tin.n, r.d[a], p2, e2);
            two_sum(p1, p2, s, es);
            float num = __fadd_rn(s, __fadd_rn(es, __fadd_rn(e1, e2)));
            q[a] = fminf(fmaxf(__fdiv_rn(num, ad), 0.f), (float)ext[a]);
        }
        th = __fdiv_rn(tin.n, ad);
        tl = __fdiv_rn(__fmaf_rn(-th, ad, tin.n), ad);
    }
    float inv[3];
    float sexit = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        inv[a] = r.sgn[a] != 0 ? 1.f / r.ad[a] : 0.f;
        if (r.sgn[a] == 0) continue;
        float farp = r.sgn[a] > 0 ? (float)ext[a] : 0.f;
        sexit = fminf(sexit, (farp - q[a]) * (float)r.sgn[a] * inv[a]);
    }
    if (!(sexit > 0.f)) return false;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float fl = floorf(q[a]);
        int ci = (int)fl;
        if (r.sgn[a] < 0 && q[a] == fl) --ci;
        c[a] = min(max(ci, 0), ext[a] - 1);
    }
    float s0 = 0.f;
    for (int it = 0; it < 16; ++it) {
        float s1 = sexit;
        int mask = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (r.sgn[a] == 0) continue;
            float plane = (float)(r.sgn[a] > 0 ? c[a] + 1 : c[a]);
            float sa = (plane - q[a]) * (float)r.sgn[a] * inv[a];
            if (sa < s1) {
                s1 = sa;
                mask = 1 << a;
            } else if (sa == s1) {
                mask |= 1 << a;
            }
        }
        if (s1 > s0) {
            CellF f;
            int below = 0, above = 0;
            corner.load8(c, f.v);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                below += f.v[k] < iso;
                above += f.v[k] > iso;
            }
            if (below != 8 && above != 8) {
                f.iso = iso;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    f.d[a] = r.d[a];
                    f.u[a] = fmaf(s0, r.d[a], q[a] - (float)c[a]);
                }
                float sig;
                if (first_root(f, s1 - s0, sig)) {
                    // depth = (t_in + s) |d|, carried in float pairs
                    float sx, ex, sy, ey, sz, ez, t1, e1, t2, e2;
                    two_prod(r.d[0], r.d[0], sx, ex);
                    two_prod(r.d[1], r.d[1], sy, ey);
                    two_prod(r.d[2], r.d[2], sz, ez);
                    two_sum(sx, sy, t1, e1);
                    two_sum(t1, sz, t2, e2);
                    float lo = ex + ey + ez + e1 + e2;
                    float rt = sqrtf(t2);
                    float rr, rre;
                    two_prod(rt, rt, rr, rre);
                    float corr = ((t2 - rr) - rre + lo) / (2.f * rt);
                    float S = tl + (s0 + sig);
                    float pp, pe;
                    two_prod(th, rt, pp, pe);
                    float depth = __fadd_rn(pp, pe + th * corr + S * (rt + corr));
                    // shade: |n . d| with n the interpolant's gradient
                    float ux = fmaf(sig, f.d[0], f.u[0]), uy = fmaf(sig, f.d[1], f.u[1]),
                          uz = fmaf(sig, f.d[2], f.u[2]);
                    const float *v = f.v;
                    float gx = lerpf(lerpf(v[1] - v[0], v[3] - v[2], uy), lerpf(v[5] - v[4], v[7] - v[6], uy), uz);
                    float gy = lerpf(lerpf(v[2] - v[0], v[3] - v[1], ux), lerpf(v[6] - v[4], v[7] - v[5], ux), uz);
                    float gz = lerpf(lerpf(v[4] - v[0], v[5] - v[1], ux), lerpf(v[6] - v[2], v[7] - v[3], ux), uy);
                    float gn = sqrtf(gx * gx + gy * gy + gz * gz);
                    float cosv = gn > 0.f ? fabsf(gx * r.d[0] + gy * r.d[1] + gz * r.d[2]) / (gn * (rt + corr)) : 0.f;
                    int grey = (int)floorf(255.f * (0.1f + 0.9f * fminf(cosv, 1.f)) + 0.5f);
                    uint32_t lc = (uint32_t)(c[0] + 4 * c[1] + 16 * c[2]);
                    payload = ((uint64_t)__float_as_uint(fmaxf(depth, 0.f)) << 20) | ((uint64_t)lc << 14) |
                              ((uint64_t)grey << 6);
                    return true;
                }
            }
        }
        if (!mask) break;
        bool out = false;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (mask >> a & 1) {
                c[a] += r.sgn[a];
                if (c[a] < 0 || c[a] >= ext[a]) out = true;
            }
        if (out) break;
        s0 = s1;
    }
    return false;
}

__global__ void __launch_bounds__(128, 4) intersect_kernel(RT R, const uint32_t *__restrict__ E,
                                                        const uint32_t *__restrict__ rbid,
                                                        const uint32_t *__restrict__ live0,
                                                        const uint32_t *__restrict__ live1,
                                                        const PassState *__restrict__ ps,
                                                        unsigned long long *keys, uint32_t *ctr, Spec S)
{
    if (ctr[C_OVERFLOW]) return;
    const uint32_t kk = ps->kk;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    const uint32_t n = ctr[C_NENT];
    const VolGeom &g = R.P.g;
    // Entries are grouped by block in block-id order, z slowest.  When the
    // first view looks down z (its central ray has d_z < 0), a ray's earlier
    // blocks have the higher ids: the queue then runs from the end, so that
    // more entries find their ray's hit already recorded and are skipped.
    bool down;
    {
        const Cam &c = R.P.views[0].cam;
        down = c.p00[2] + 0.5f * (float)R.P.W * c.du[2] + 0.5f * (float)R.P.H * c.dv[2] < 0.f;
    }
    for (;;) {
        const uint32_t base = warp_take(&ctr[C_QISECT]);
        if (base >= n) break;
        const uint32_t q = base + (threadIdx.x & 31);
        if (q >= n) continue;
        const uint32_t idx = down ? n - 1 - q : q;
        uint32_t e = E[idx];
        uint32_t b = rbid[e];
        uint32_t i, j;
        if (S.koff) {
            i = S.eray[e];
            j = e - S.koff[i];
        } else {
            i = e / kk;
            j = e - i * kk;
        }
        uint32_t ray = live[i];
        // a hit already recorded from an earlier block of this ray (smaller
        // j) wins the atomicMin whatever this block holds
        if ((uint32_t)(__ldcg(keys + ray) >> 52) < j) continue;
        Ray r;
        int view, px, py;
        ray_pixel(R.P, ray, view, px, py);
        const View &vw = R.P.views[view];
        const float iso = vw.iso;
        make_ray(r, vw.cam.eye, vw.cam.p00, vw.cam.du, vw.cam.dv, px, py);
        int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]), bz = (int)(b / ((uint32_t)g.nb[0] * g.nb[1]));
        GlobalCorners gc;
        gc.cache = R.cache;
        {
            int ext[3];
            block_extent(g, bx, by, bz, ext);
            neighbour_slots(R, bx, by, bz, ext, gc.slots);
        }
        uint64_t payload;
        if (intersect_block(R, r, iso, bx, by, bz, gc, payload)) atomicMin(keys + ray, ((uint64_t)j << 52) | payload);
    }
}

// The intersection with each block's dual grid staged in shared memory, as
// Sec. 3.7's work groups do: a warp takes 32 entries from the queue (entries
// are grouped by block, so their blocks form runs), copies the 5^3 values of
// each distinct block among them from the cache slots into shared memory
// (4 values per lane and block), then intersects its entries reading corners
// from there.  Same arithmetic on the same values as intersect_kernel, so the
// same keys.  It pays when blocks carry several entries each (one staging
// serves them all); the per-cell loads of intersect_kernel touch only the
// corners of the cells a ray crosses.
constexpr int kStageWarps = 3;   // 3 x 16 KB: the static shared-memory limit

__global__ void __launch_bounds__(32 * kStageWarps, 4) intersect_staged_kernel(
    RT R, const uint32_t *__restrict__ E, const uint32_t *__restrict__ rbid, const uint32_t *__restrict__ live0,
    const uint32_t *__restrict__ live1, const PassState *__restrict__ ps, unsigned long long *keys, uint32_t *ctr,
    Spec S)
{
    __shared__ float s_grid[kStageWarps][32][128];
    if (ctr[C_OVERFLOW]) return;
    const uint32_t kk = ps->kk;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    const uint32_t n = ctr[C_NENT];
    const VolGeom &g = R.P.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        const uint32_t base = warp_take(&ctr[C_QISECT]);
        if (base >= n) break;
        const uint32_t idx = base + lane;
        const bool valid = idx < n;
        const uint32_t e = valid ? E[idx] : 0u;
        const uint32_t b = valid ? rbid[e] : kNone;
        const uint32_t bprev = __shfl_up_sync(0xFFFFFFFFu, b, 1);
        const bool start = valid && (lane == 0 || b != bprev);
        const unsigned starts = __ballot_sync(0xFFFFFFFFu, start);
        const int my_g = __popc(starts & ((2u << lane) - 1u)) - 1;   // this entry's block among the warp's
        // stage the distinct blocks, one after another
        unsigned rem = starts;
        for (int gi = 0; rem; ++gi) {
            const int src = __ffs(rem) - 1;
            rem &= rem - 1u;
            const uint32_t bg = __shfl_sync(0xFFFFFFFFu, b, src);
            const int bx = (int)(bg % g.nb[0]), by = (int)((bg / g.nb[0]) % g.nb[1]),
                      bz = (int)(bg / ((uint32_t)g.nb[0] * g.nb[1]));
            int ext[3];
            block_extent(g, bx, by, bz, ext);
            uint32_t my_slot = 0u;
            if (lane < 8) {
                const int k = lane;
                const int x = bx + (k & 1), y = by + ((k >> 1) & 1), z = bz + (k >> 2);
                const bool need = (!(k & 1) || ext[0] == 4) && (!(k & 2) || ext[1] == 4) && (!(k & 4) || ext[2] == 4);
                my_slot = (need && x < g.nb[0] && y < g.nb[1] && z < g.nb[2])
                              ? R.blk_slot[x + (int64_t)g.nb[0] * (y + (int64_t)g.nb[1] * z)]
                              : 0u;
            }
            float *dst = s_grid[w][gi];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int q = lane + 32 * t;
                const int lx = q % 5, ly = (q / 5) % 5, lz = q / 25;
                const int nsel = (lx >> 2) | ((ly >> 2) << 1) | ((lz >> 2) << 2);
                const uint32_t slot = __shfl_sync(0xFFFFFFFFu, my_slot, nsel);
                // corners the block's cells can reach: up to ext along each axis
                if (q < 125 && lx <= ext[0] && ly <= ext[1] && lz <= ext[2])
                    dst[q] = __ldg(R.cache + (uint64_t)slot * 64 + (lx & 3) + 4 * (ly & 3) + 16 * (lz & 3));
            }
        }
        __syncwarp();
        if (valid) {
            uint32_t i, j;
            if (S.koff) {
                i = S.eray[e];
                j = e - S.koff[i];
            } else {
                i = e / kk;
                j = e - i * kk;
            }
            const uint32_t ray = live[i];
            // a hit already recorded from an earlier block of this ray wins
            if ((uint32_t)(__ldcg(keys + ray) >> 52) >= j) {
                Ray r;
                int view, px, py;
                ray_pixel(R.P, ray, view, px, py);
                const View &vw = R.P.views[view];
                make_ray(r, vw.cam.eye, vw.cam.p00, vw.cam.du, vw.cam.dv, px, py);
                const int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]),
                          bz = (int)(b / ((uint32_t)g.nb[0] * g.nb[1]));
                uint64_t payload;
                if (intersect_block(R, r, vw.iso, bx, by, bz, SharedCorners{s_grid[w][my_g]}, payload))
                    atomicMin(keys + ray, ((uint64_t)j << 52) | payload);
            }
        }
        __syncwarp();   // the staging area is rewritten by the next take
    }
}

// ---------------------------------------------------------------- resolve
// Resolve, one thread per live position i < n_live: a ray with a key writes
// its hit, a ray whose walk left the volume its miss; every other ray stays
// live.  Bit i of `alive` (warp ballots) marks the survivors.
__global__ void __launch_bounds__(256) resolve_kernel(const uint32_t *__restrict__ live0,
                                                      const uint32_t *__restrict__ live1,
                                                      const PassState *__restrict__ ps, int Dx, int Dy, VolGeom g,
                                                      unsigned long long *__restrict__ keys,
                                                      const uint32_t *__restrict__ rbid,
                                                      uint64_t *__restrict__ state_in,
                                                      const uint64_t *__restrict__ state_out,
                                                      uint8_t *__restrict__ status, float *__restrict__ depth,
                                                      uint32_t *__restrict__ rgba, uint32_t *__restrict__ block,
                                                      uint64_t *__restrict__ cell, int32_t *__restrict__ final_pass,
                                                      uint32_t *__restrict__ alive_bits, uint32_t *ctr, Spec S,
                                                      Trace T)
{
    if (ctr[C_OVERFLOW]) return;
    const uint32_t *live = (ps->parity & 1) ? live1 : live0;
    const uint32_t n_live = ps->n_live, nproc = ps->nproc, kk = ps->kk;
    const int64_t n_pad = (int64_t)ps->live_words * 32;
    const int pass = (int)ps->pass + 1;
    uint32_t nh = 0, ng = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x) {   // whole warps iterate
        bool alive = i < (int64_t)n_live;
        if (i < (int64_t)nproc) {
            const uint32_t ray = live[i];
            const unsigned long long key = keys[ray];
            const uint64_t st = state_out[ray];
            state_in[ray] = st;
            if (key != kNoKey) {
                uint32_t j = (uint32_t)(key >> 52);
                uint32_t b = rbid[(S.koff ? (uint64_t)S.koff[i] : (uint64_t)i * kk) + j];
                uint32_t lc = (uint32_t)((key >> 14) & 63u), grey = (uint32_t)((key >> 6) & 255u);
                int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]),
                    bz = (int)(b / ((uint32_t)g.nb[0] * g.nb[1]));
                uint64_t cx = 4 * bx + (lc & 3), cy = 4 * by + ((lc >> 2) & 3), cz = 4 * bz + (lc >> 4);
                depth[ray] = __uint_as_float((uint32_t)((key >> 20) & 0xFFFFFFFFull));
                rgba[ray] = grey | (grey << 8) | (grey << 16) | (255u << 24);
                block[ray] = b;
                cell[ray] = cx + (uint64_t)Dx * (cy + (uint64_t)Dy * cz);
                final_pass[ray] = pass;
                status[ray] = 1;
                keys[ray] = kNoKey;
                alive = false;
                ++nh;
                if (T.taken) T.need[ray] = T.taken[ray] + j + 1u;
            } else if ((st >> 48) & kDone) {
                final_pass[ray] = pass;
                status[ray] = 2;
                alive = false;
                ++ng;
                if (T.taken) {
                    const uint64_t off = S.koff ? S.koff[i] : (uint64_t)i * kk;
                    const uint32_t ki = S.koff ? S.kray[i] : kk;
                    uint32_t c = 0;
                    for (uint32_t q = 0; q < ki; ++q) c += rbid[off + q] != kNone;
                    T.need[ray] = T.taken[ray] + c;
                }
            } else if (T.taken) {
                // live on: it took exactly its count of visible blocks
                T.taken[ray] += S.koff ? S.kray[i] : kk;
            }
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, alive);
        if ((threadIdx.x & 31) == 0) alive_bits[i >> 5] = bits;
    }
    nh = __reduce_add_sync(0xFFFFFFFFu, nh);
    ng = __reduce_add_sync(0xFFFFFFFFu, ng);
    if ((threadIdx.x & 31) == 0) {
        if (nh) atomicAdd(&ctr[C_HIT], nh);
        if (ng) atomicAdd(&ctr[C_MISSRAY], ng);
    }
}

// the next live list from the alive bitmap, in order
struct LiveEmit {
    uint32_t *live0, *live1;
    const PassState *ps;
    __device__ void operator()(int64_t i, uint32_t pre, uint32_t c) const
    {
        if (!c) return;
        if (ps->parity & 1) live0[pre] = live1[i];
        else live1[pre] = live0[i];
    }
};

// ----------------------------------------------------- per-ray speculation
__host__ __device__ inline bool per_ray_mode(uint32_t mode)
{
    return mode == SPR_SPEC_HASHED || mode == SPR_SPEC_LEARNED;
}

// SPR_SPEC_HASHED: live position i takes k = 1 + h(ray, pass) mod k_max
// (capped by the attempt's kk), a deterministic per-ray count that exercises
// the per-ray entry layout with no model.
__global__ void hashed_k_kernel(const uint32_t *__restrict__ live0, const uint32_t *__restrict__ live1,
                                const PassState *__restrict__ ps, uint32_t *__restrict__ kray)
{
    const uint32_t nproc = ps->nproc, kk = ps->kk, kmax = ps->k_max, pass = ps->pass;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nproc; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = live[i] * 0x9E3779B1u ^ (pass + 1u) * 0x85EBCA77u;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        kray[i] = min(kk, 1u + h % kmax);
    }
}

// The 12 features of a live ray for the speculation policy (all in [0, 1]
// or [-1, 1]): pass index / 8; the current block's position in the block
// grid (3); the unit ray direction (3); the distance from the eye to the
// current block's centre over the volume diagonal (how far the ray has
// come); the fraction of occupied blocks in its coarse cell and of occupied
// coarse cells in its super cell (the occupancy ahead); the isovalue; the
// fraction of rays still live.
__device__ __noinline__ void ray_features(const Geo &P, const PassState *ps, uint32_t ray, uint64_t st,
                                          float f[mlp::kIn])
{
    const VolGeom &g = P.g;
    int view, px, py;
    ray_pixel(P, ray, view, px, py);
    const View &vw = P.views[view];
    Ray r;
    make_ray(r, vw.cam.eye, vw.cam.p00, vw.cam.du, vw.cam.dv, px, py);
    int b0 = (int)(st & 0xFFFF), b1 = (int)((st >> 16) & 0xFFFF), b2 = (int)((st >> 32) & 0xFFFF);
    if ((st >> 48) & kBoxed) {
        // a walk not yet started from the occupied box: the features are
        // those of the block where the ray enters the volume
        Tq tin{0.f, 1.f};
        for (int a = 0; a < 3; ++a) {
            if (r.sgn[a] == 0) continue;
            const Tq tn = plane_t(r, a, r.sgn[a] > 0 ? 0.f : (float)(g.dims[a] - 1));
            if (tcmp(tn, tin) > 0) tin = tn;
        }
        b0 = locate_block(r, 0, tin, g.tb[0]);
        b1 = locate_block(r, 1, tin, g.tb[1]);
        b2 = locate_block(r, 2, tin, g.tb[2]);
    }
    const float dn = sqrtf(r.d[0] * r.d[0] + r.d[1] * r.d[1] + r.d[2] * r.d[2]);
    const float ex = (float)(g.dims[0] - 1), ey = (float)(g.dims[1] - 1), ez = (float)(g.dims[2] - 1);
    const float diag = sqrtf(ex * ex + ey * ey + ez * ez);
    const float cx = 4.f * b0 + 2.f - r.e[0], cy = 4.f * b1 + 2.f - r.e[1], cz = 4.f * b2 + 2.f - r.e[2];
    const uint32_t c = (uint32_t)(b0 >> 2) + (uint32_t)g.nc[0] * ((uint32_t)(b1 >> 2) + (uint32_t)g.nc[1] * (uint32_t)(b2 >> 2));
    const uint32_t sc = (uint32_t)(b0 >> 4) + (uint32_t)P.occ.ns[0] * ((uint32_t)(b1 >> 4) + (uint32_t)P.occ.ns[1] * (uint32_t)(b2 >> 4));
    f[0] = 0.125f * (float)ps->pass;
    f[1] = (b0 + 0.5f) / (float)g.tb[0];
    f[2] = (b1 + 0.5f) / (float)g.tb[1];
    f[3] = (b2 + 0.5f) / (float)g.tb[2];
    f[4] = r.d[0] / dn;
    f[5] = r.d[1] / dn;
    f[6] = r.d[2] / dn;
    f[7] = sqrtf(cx * cx + cy * cy + cz * cz) / diag;
    f[8] = (float)__popcll(P.occ.fmask[view * P.fstride + c]) * (1.f / 64.f);
    f[9] = (float)__popcll(P.occ.smask[view * P.sstride + sc]) * (1.f / 64.f);
    f[10] = vw.iso;
    f[11] = (float)ps->n_live / (float)max(ps->npix, 1u);
}

// Speculation count of a ray: the policy's upper-quantile estimate of the
// log2 of the visible blocks it still needs, k = ceil(2^(y1 + margin)) in
// [1, 32]; in the passes the floor applies to (all with SPR_POLICY_FLOOR,
// all but the first with SPR_POLICY_FLOOR_AFTER_FIRST) never below the
// paper's uniform count for the pass (min(k_max, floor(w*h / N_Act)), Sec. 4);
// capped at `cap`.
constexpr uint32_t kLearnedMax = 32;
__device__ __forceinline__ uint32_t policy_k(float y, float margin, uint32_t floor_k, uint32_t cap)
{
    const float z = fminf(fmaxf(y + margin, -1.f), 12.f);
    const uint32_t k = min(kLearnedMax, max(1u, (uint32_t)ceilf(exp2f(z))));
    return min(cap, max(k, floor_k));
}

// SPR_SPEC_LEARNED: features of 128 live rays per tile, the policy MLP on
// the tensor cores (mlp.cuh), each ray's count.  params holds the fp32
// parameter vector, the margin and the first floored pass.  Persistent CTAs
// over the tiles.
__global__ void __launch_bounds__(128) policy_kernel(Geo P, const uint32_t *__restrict__ live0,
                                                     const uint32_t *__restrict__ live1,
                                                     const PassState *__restrict__ ps,
                                                     const uint64_t *__restrict__ state_in,
                                                     const float *__restrict__ params, uint32_t *__restrict__ kray,
                                                     uint32_t *ctr)
{
    __shared__ mlp::Smem S;
    const uint32_t nproc = ps->nproc;
    const int64_t ntiles = ((int64_t)nproc + mlp::kRows - 1) / mlp::kRows;
    if ((int64_t)blockIdx.x >= ntiles) return;   // uniform per CTA: no TMEM taken
    const float margin = params[mlp::kParams];
    const uint32_t cap = min(ps->kk, ps->k_max);
    // params[kParams + 1]: the first pass (0-based) whose counts are floored
    // at the paper's uniform count; negative: never
    const float floor_from = params[mlp::kParams + 1];
    const uint32_t floor_k = (floor_from >= 0.f && (float)ps->pass >= floor_from)
                                 ? max(1u, min(ps->k_max, ps->npix / max(ps->n_live, 1u)))
                                 : 1u;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    if (floor_k >= kLearnedMax) {
        // the floor is at least any count the policy can give: no inference
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nproc;
             i += (int64_t)gridDim.x * blockDim.x)
            kray[i] = min(cap, floor_k);
        return;
    }
    mlp::tile_setup(S, params);
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * mlp::kRows + threadIdx.x;
        float f[mlp::kIn];
        if (i < nproc) {
            const uint32_t ray = live[i];
            ray_features(P, ps, ray, state_in[ray], f);
        } else {
#pragma unroll
            for (int q = 0; q < mlp::kIn; ++q) f[q] = 0.f;
        }
        mlp::store_features(S, f);
        float y[mlp::kOut];
        if (!mlp::forward_tile(S, phase, y)) {
            if (threadIdx.x == 0) atomicOr(&ctr[C_BAD], 8u);
            // every ray of the remaining tiles still gets a count
            for (int64_t t2 = tile; t2 < ntiles; t2 += gridDim.x) {
                const int64_t i2 = t2 * mlp::kRows + threadIdx.x;
                if (i2 < nproc) kray[i2] = 1u;
            }
            break;
        }
        if (i < nproc) kray[i] = policy_k(y[1], margin, floor_k, cap);
    }
    mlp::tile_teardown(S);
}

__device__ __forceinline__ bool trace_pick(uint32_t ray, uint32_t mod)
{
    uint32_t h = ray * 0x9E3779B1u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    return mod <= 1 || h % mod == 0;
}

__global__ void __launch_bounds__(128) trace_kernel(Geo P, const uint32_t *__restrict__ live0,
                                                    const uint32_t *__restrict__ live1,
                                                    const PassState *__restrict__ ps,
                                                    const uint64_t *__restrict__ state_in, Trace T)
{
    if (ps->retries != 0) return;   // one sample per ray and pass (the first attempt)
    const uint32_t n = ps->n_live;
    const uint32_t *__restrict__ live = (ps->parity & 1) ? live1 : live0;
    const bool first = ps->pass == 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t ray = live[i];
        if (first) {
            T.taken[ray] = 0u;
            T.need[ray] = 0u;
        }
        if (!trace_pick(ray, T.mod)) continue;
        const uint32_t slot = atomicAdd(T.count, 1u);
        if (slot >= T.cap) continue;
        float f[mlp::kIn];
        ray_features(P, ps, ray, state_in[ray], f);
#pragma unroll
        for (int q = 0; q < mlp::kIn; ++q) T.feat[(uint64_t)slot * mlp::kIn + q] = f[q];
        T.ray[slot] = ray;
        T.cons[slot] = first ? 0u : T.taken[ray];
    }
}

// labels of samples [from, min(count, cap)): the visible blocks the ray
// still needed at the sample = need - taken then, at least 1
__global__ void trace_label_kernel(Trace T, uint32_t from, uint32_t *__restrict__ labels)
{
    const uint32_t n = min(*T.count, T.cap);
    for (int64_t s = (int64_t)from + blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t need = T.need[T.ray[s]], c = T.cons[s];
        labels[s] = need > c ? need - c : 1u;
    }
}

// ------------------------------------------------------------ pass control
__global__ void begin_pass_kernel(PassState *ps, uint32_t *ctr)
{
    if (threadIdx.x < C_COUNT) ctr[threadIdx.x] = 0u;
    if (threadIdx.x == 0 && !ps->open) {
        uint32_t n = ps->n_live;
        // per-ray modes: kk caps every ray's own count (halved on overflow)
        uint32_t k = ps->spec_mode == SPR_SPEC_FIXED
                         ? ps->k_fixed
                         : (ps->spec_mode == SPR_SPEC_ADAPTIVE ? max(1u, min(ps->k_max, ps->npix / max(n, 1u)))
                                                                : ps->k_max);
        ps->k = k;
        ps->kk = k;
        ps->nproc = n;
        ps->retries = 0;
        ps->live_words = (n + 31) / 32;
    }
}

// ends an attempt; `recs` and `mirror` live in mapped host memory, so the
// host reads the pass state and records after one stream synchronisation
__global__ void end_pass_kernel(PassState *ps, const uint32_t *ctr, spr_pass_stats *recs, uint32_t n_recs,
                                PassState *mirror, cudaGraphConditionalHandle handle, int use_handle)
{
    if (threadIdx.x != 0) return;
    if (ps->n_live > 0) ps->attempts += 1;
    if (ctr[C_SCANFLAGS] || ctr[C_BAD]) {
        ps->error = (ctr[C_SCANFLAGS] ? 1u : 0u) | (ctr[C_BAD] << 1);
        ps->run = 0;
    } else if (ps->n_live == 0) {
        ps->run = 0;
    } else if (ctr[C_OVERFLOW]) {
        ps->retries += 1;
        ps->open = 1;
        if (ps->kk > 1) ps->kk /= 2;
        else ps->nproc = max(1u, ps->nproc / 2);
    } else {
        ps->tot_decoded += ctr[C_NMISS];
        ps->tot_entries += ctr[C_NENT];
        ps->tot_evicted += ctr[C_EVICT];
        ps->tot_hits += ctr[C_HIT];
        if (ps->pass < n_recs) {
            spr_pass_stats st{};
            st.pass = (int32_t)ps->pass + 1;
            st.k = (int32_t)ps->k;
            st.k_used = (int32_t)ps->kk;
            st.retries = (int32_t)ps->retries;
            st.n_active = ps->n_live;
            st.n_processed = ps->nproc;
            st.n_entries = ctr[C_NENT];
            st.n_visible = ctr[C_NVIS];
            st.n_requested = ctr[C_NACT];
            st.n_decoded = ctr[C_NMISS];
            st.n_evicted = ctr[C_EVICT];
            st.n_term_hit = ctr[C_HIT];
            st.n_term_miss = ctr[C_MISSRAY];
            st.n_active_after = ctr[C_NLIVE];
            st.utilization = (double)ctr[C_NENT] / (double)ps->npix;
            st.n_steps = ctr[C_STEPS];
            st.max_steps = ctr[C_MAXSTEPS];
            recs[ps->pass] = st;
        }
        ps->n_used += ps->fresh_hi - ps->fresh_lo;
        ps->fresh_lo = ps->fresh_hi;
        ps->pass += 1;
        ps->parity ^= 3u;
        ps->n_live = ctr[C_NLIVE];
        ps->open = 0;
        ps->run = (ps->n_live > 0 && ps->pass < ps->max_passes) ? 1u : 0u;
    }
    *mirror = *ps;
    if (use_handle) cudaGraphSetConditional(handle, ps->run);
}

// Empty the cache by undoing only what was used: every slot below
// max(fresh_lo, fresh_hi) (slots above were never handed out) drops its
// block's mapping and its touched flag; then every slot is fresh again.
// Runs when `reset` is null or *reset is nonzero.
__global__ void cache_clear_used_kernel(PassState *ps, const uint32_t *reset, uint32_t *__restrict__ slot_blk,
                                        uint32_t *__restrict__ blk_slot, uint8_t *__restrict__ touched,
                                        int64_t n_slots)
{
    if (reset && !*reset) return;
    const int64_t hi = min((int64_t)max(ps->fresh_lo, ps->fresh_hi), n_slots);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = slot_blk[i];
        if (b != kNone) {
            blk_slot[b] = kNone;
            slot_blk[i] = kNone;
        }
        touched[i] = 0;
    }
}

// First kernel of a render's start graph: the speculation settings, zeroed
// pass counters, and (when p->reset) the used slots emptied.  The LRU state
// itself is reset by a later kernel, after every thread here has read it.
__global__ void start_kernel(PassState *ps, const DevParams *p, uint32_t *ctr, uint32_t *__restrict__ slot_blk,
                             uint32_t *__restrict__ blk_slot, uint8_t *__restrict__ touched, int64_t n_slots)
{
    if (blockIdx.x == 0) {
        if (threadIdx.x < C_COUNT) ctr[threadIdx.x] = 0u;
        if (threadIdx.x == 0) {
            ps->spec_mode = p->spec_mode;
            ps->k_fixed = p->k_fixed;
            ps->k_max = p->k_max;
            ps->npix = p->npix;
            ps->coop_below = p->coop_below;
            ps->seg_threads = p->seg_threads;
        }
    }
    if (!p->reset) return;
    const int64_t hi = min((int64_t)max(ps->fresh_lo, ps->fresh_hi), n_slots);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = slot_blk[i];
        if (b != kNone) {
            blk_slot[b] = kNone;
            slot_blk[i] = kNone;
        }
        touched[i] = 0;
    }
}

__global__ void cache_reset_kernel(PassState *ps, const uint32_t *reset)
{
    if (threadIdx.x != 0 || (reset && !*reset)) return;
    lru_reset(ps);
}

__global__ void config_kernel(PassState *ps, const DevParams *p)
{
    if (threadIdx.x != 0) return;
    ps->spec_mode = p->spec_mode;
    ps->k_fixed = p->k_fixed;
    ps->k_max = p->k_max;
    ps->npix = p->npix;
    ps->coop_below = p->coop_below;
    ps->seg_threads = p->seg_threads;
}

// after ray generation: the live list is list 0 and the pass count restarts
__global__ void after_raygen_kernel(PassState *ps, const uint32_t *ctr, PassState *mirror, const uint32_t *more_dev)
{
    if (threadIdx.x != 0) return;
    ps->n_live = ctr[C_NLIVE];
    ps->n_enter = ctr[C_NLIVE];
    ps->pass = 0;
    ps->parity &= ~1u;
    ps->open = 0;
    ps->retries = 0;
    ps->attempts = 0;
    ps->tot_decoded = ps->tot_entries = ps->tot_evicted = ps->tot_hits = 0ull;
    ps->error = ctr[C_SCANFLAGS] ? 1u : 0u;
    ps->run = ps->n_live > 0 ? 1u : 0u;
    if (more_dev) {   // the pass limit of this call
        ps->max_passes = ps->pass + *more_dev;
        ps->run = (ps->n_live > 0 && *more_dev > 0) ? 1u : 0u;
    }
    *mirror = *ps;
}

// -------------------------------------------------------------- utilities
thread_local int64_t *g_launch_counter = nullptr;
inline void count_launch(int n = 1)
{
    if (g_launch_counter) *g_launch_counter += n;
}

template <class CF, class EF>
int run_compact(DevBuf &status, DevBuf &ticket, uint32_t *flags, int64_t n_cap, const uint32_t *n_dev,
                CF cf, EF ef, uint32_t *total, cudaStream_t s, int64_t spin = kDefaultSpinLimit,
                int64_t withhold = -1, uint32_t *over = nullptr, uint32_t over_limit = 0)
{
    int64_t tiles = std::max<int64_t>(1, scan_tiles(n_cap));
    if ((size_t)tiles * sizeof(unsigned long long) > status.bytes)
        return set_error(SPR_ERR_INVALID_ARG, "scan of %lld items exceeds its scratch", (long long)n_cap);
    // status words and ticket/done/epoch were zeroed when allocated; the
    // kernel leaves them ready for the next launch
    ScanCtl ctl{status.as<unsigned long long>(), (int64_t)(status.bytes / sizeof(unsigned long long)),
                ticket.as<unsigned int>(), flags, spin, withhold, over, over_limit};
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)device_sm_count() * 4);
    compact_kernel<CF, EF><<<(unsigned)grid, kScanThreads, 0, s>>>(n_cap, n_dev, ctl, cf, ef, total);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    return SPR_OK;
}

// compaction of a block bitmap of nwords words (two kernels); tsum holds
// bits_tiles(nwords) counts
template <class EF>
int run_bits_compact(uint32_t *bits, int64_t nwords, uint32_t *tsum, EF ef, uint32_t *total, cudaStream_t s,
                     uint32_t *over = nullptr, uint32_t over_limit = 0, bool clear = false)
{
    const int64_t tiles = bits_tiles(nwords);
    bits_reduce_kernel<<<(unsigned)tiles, kBitsThreads, 0, s>>>(bits, nwords, tsum);
    bits_emit_kernel<EF><<<(unsigned)tiles, kBitsThreads, 0, s>>>(bits, nwords, tsum, ef, total, over, over_limit,
                                                                  clear);
    count_launch(2);
    SPR_CUDA_TRY(cudaGetLastError());
    return SPR_OK;
}

}  // namespace spr

using namespace spr;

// ================================================================= renderer
struct spr_renderer {
    spr_volume *vol = nullptr;
    int W = 0, H = 0;
    int64_t npix = 0;             // rays of the active views: n_views * W * H
    int n_views = 1;              // active views (views >= n_views generate no rays)
    int view_cap = 1;             // views the buffers and captured graphs are sized for
    int64_t npix_cap = 0;         // view_cap * W * H
    View views[kMaxViews] = {};   // camera and isovalue per view
    uint64_t cam_set = 0;         // bit v: view v has a camera
    float iso = 0.5f;             // isovalue given to views by spr_set_isovalue
    int spec_mode = SPR_SPEC_ADAPTIVE, k_fixed = 1, k_max = 64;
    uint32_t coop_below = kCoopBelowDefault;
    uint32_t seg_threads = kSegThreadsDefault;
    bool isect_staged = false;    // intersect_staged_kernel instead of intersect_kernel
    int64_t n_slots = 0;
    bool profiling = false;

    int grid_isect = 1;   // one wave of the work-queue kernel
    bool need_raygen = true;
    bool cache_dirty = true;
    bool cache_init = false;    // slot tables consistent (else the next reset clears them whole)
    bool bits_dirty = false;    // a render stopped on a device error: clear the bitmaps
    bool params_dirty = true;   // camera / isovalue / speculation not yet on the device
    int pass = 0;               // passes completed (host mirror of the device state)
    uint32_t n_live = 0;
    uint32_t n_enter = 0;
    float ms_raygen = 0.f;

    DevBuf state_in, state_out, status, live[2], keys;
    DevBuf fb_depth, fb_rgba, fb_block, fb_cell, fb_final;
    DevBuf rbid, erank, E;
    DevBuf kray, koff, eray;      // per-ray speculation (Spec)
    bool policy_set = false;      // a policy MLP is loaded (SPR_SPEC_LEARNED)
    DevBuf policy;                // fp32 parameters + margin
    // training traces (spr_set_trace): caller buffers, per-ray bookkeeping
    bool tracing = false;
    float *tr_feat = nullptr;
    uint32_t *tr_ray = nullptr, *tr_cons = nullptr;
    uint32_t tr_cap = 0, tr_mod = 1, tr_from = 0;
    DevBuf tr_count, tr_taken, tr_need;
    int64_t cap_entries = 0;
    DevBuf vis_bits, act_bits, vis_wpre, ivis, iact, nbrays, obrays;
    DevBuf bits_tsum;   // tile counts of the two bitmap compactions (active, visible)
    DevBuf lbits;   // enter bits at ray generation, alive bits at resolve (one per live position)
    int64_t nwords = 0, cap_act = 0;
    DevBuf cache, blk_slot, slot_blk, lru[2], touched, miss, victim;
    int64_t launches = 0;         // kernels launched since the last render started
    DevBuf occ_fine, occ_super;   // brick masks per coarse cell and per super cell
    DevBuf occ_box;               // occupied box per view (8 ints)
    Occ occ{};
    float occ_iso[kMaxViews];     // isovalue each view's brick masks were built for
    // look-back scratch, one set per branch of a pass that can run a scan
    // while another branch runs one: [0] main (grouping, resolve, ray
    // generation), [1] cache, [2] LRU order
    DevBuf scan_status[3], scan_ticket[3];
    DevBuf ctr;
    DevBuf ps, camd;              // device pass state, DevParams
    // mapped host memory written by the device: per-pass records and a copy
    // of the pass state after each pass (host pointers h_*, device aliases d_*)
    spr_pass_stats *h_recs = nullptr, *d_recs = nullptr;
    PassState *d_hps = nullptr;
    DevParams *h_params = nullptr;  // pinned source of camd
    cudaEvent_t ev_upload = nullptr;  // the last copy out of h_params has run
    cudaGraphExec_t gstart = nullptr, glimit = nullptr;  // render start with / without ray generation
    static constexpr int kRecCap = 4096;
    PassState *h_ps = nullptr;    // mapped (see d_hps)
    uint32_t *h_ctr = nullptr;    // pinned
    cudaEvent_t ev[8] = {};
    // fork/join of the pass's branches (no timing)
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t jev[5] = {};
    // the pass loop as one graph: a while node whose body is one pass
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gprof = nullptr;  // one attempt with event nodes between stages
    int graph_kernels = 0;        // kernels in one pass of the body
    uint64_t graph_gen = 0;       // counts drop_graph calls (a batch's captured copies go stale with them)
    // a render enqueued by spr_render_submit and not yet collected
    bool busy = false;
    cudaStream_t sub_stream = nullptr;
    bool sub_fresh = false;
    int sub_first = 0;            // passes completed before the submitted render
    PassState sub_before{};       // pass state before it (totals of a continued render)
};

namespace {

void drop_graph(spr_renderer *r)
{
    ++r->graph_gen;
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    if (r->graph) cudaGraphDestroy(r->graph);
    if (r->gprof) cudaGraphExecDestroy(r->gprof);
    if (r->gstart) cudaGraphExecDestroy(r->gstart);
    if (r->glimit) cudaGraphExecDestroy(r->glimit);
    r->gprof = nullptr;
    r->gexec = nullptr;
    r->graph = nullptr;
    r->gstart = nullptr;
    r->glimit = nullptr;
}

void free_all(spr_renderer *r)
{
    cudaDeviceSynchronize();
    drop_graph(r);
    DevBuf *bufs[] = {&r->state_in, &r->state_out, &r->status, &r->live[0], &r->live[1], &r->keys,
                      &r->fb_depth, &r->fb_rgba, &r->fb_block, &r->fb_cell, &r->fb_final, &r->rbid,
                      &r->erank, &r->E, &r->vis_bits, &r->act_bits, &r->vis_wpre, &r->bits_tsum,
                      &r->ivis, &r->iact, &r->nbrays, &r->obrays, &r->cache, &r->blk_slot,
                      &r->slot_blk, &r->lru[0], &r->lru[1], &r->touched, &r->miss, &r->victim,
                      &r->scan_status[0], &r->scan_status[1], &r->scan_status[2], &r->scan_ticket[0],
                      &r->scan_ticket[1], &r->scan_ticket[2], &r->ctr, &r->occ_fine, &r->occ_super,
                      &r->occ_box, &r->ps, &r->camd, &r->lbits, &r->kray, &r->koff, &r->eray, &r->policy,
                      &r->tr_count, &r->tr_taken, &r->tr_need};
    for (DevBuf *b : bufs) buf_free(*b, nullptr);
    if (r->h_ctr) cudaFreeHost(r->h_ctr);
    if (r->h_ps) cudaFreeHost(r->h_ps);
    if (r->h_recs) cudaFreeHost(r->h_recs);
    r->h_recs = r->d_recs = nullptr;
    r->d_hps = nullptr;
    if (r->h_params) cudaFreeHost(r->h_params);
    r->h_params = nullptr;
    if (r->ev_upload) cudaEventDestroy(r->ev_upload);
    r->ev_upload = nullptr;
    r->h_ctr = nullptr;
    r->h_ps = nullptr;
    for (auto &e : r->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : r->jev)
        if (e) cudaEventDestroy(e);
    for (auto &a : r->aux)
        if (a) cudaStreamDestroy(a);
    if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
    r->cap_stream = nullptr;
}

int64_t entries_needed(const spr_renderer *r)
{
    int64_t k = r->spec_mode == SPR_SPEC_FIXED ? r->k_fixed : (per_ray_mode(r->spec_mode) ? r->k_max : 1);
    return std::max<int64_t>(1, r->npix_cap * k);
}

int ensure_entry_buffers(spr_renderer *r, cudaStream_t s)
{
    int64_t cap = entries_needed(r);
    if (cap > 0x7FFFFFFFll)
        return set_error(SPR_ERR_INVALID_ARG, "width*height*k = %lld exceeds 2^31 entries", (long long)cap);
    if (per_ray_mode(r->spec_mode) &&
        (r->eray.bytes < sizeof(uint32_t) * (size_t)std::max(cap, r->cap_entries) ||
         r->kray.bytes < sizeof(uint32_t) * (size_t)r->npix_cap)) {
        drop_graph(r);
        SPR_TRY(buf_reserve(r->eray, sizeof(uint32_t) * std::max(cap, r->cap_entries), s));
        SPR_TRY(buf_reserve(r->kray, sizeof(uint32_t) * r->npix_cap, s));
        SPR_TRY(buf_reserve(r->koff, sizeof(uint32_t) * r->npix_cap, s));
    }
    if (cap <= r->cap_entries) return SPR_OK;
    drop_graph(r);
    SPR_TRY(buf_reserve(r->rbid, sizeof(uint32_t) * cap, s));
    SPR_TRY(buf_reserve(r->erank, sizeof(uint32_t) * cap, s));
    SPR_TRY(buf_reserve(r->E, sizeof(uint32_t) * cap, s));
    SPR_TRY(buf_reserve(r->ivis, sizeof(uint32_t) * cap, s));
    SPR_TRY(buf_reserve(r->nbrays, sizeof(uint32_t) * (cap + 1), s));
    SPR_TRY(buf_reserve(r->obrays, sizeof(uint32_t) * (cap + 1), s));
    int64_t act = std::min<int64_t>(r->vol->g.nblocks, 8 * cap);
    SPR_TRY(buf_reserve(r->iact, sizeof(uint32_t) * act, s));
    SPR_TRY(buf_reserve(r->miss, sizeof(uint32_t) * act, s));
    SPR_TRY(buf_reserve(r->victim, sizeof(uint32_t) * act, s));
    r->cap_act = act;
    r->cap_entries = cap;
    return SPR_OK;
}

int ensure_scan_scratch(spr_renderer *r, cudaStream_t s)
{
    int64_t biggest = std::max({tiled_ray_count(r->W, r->H) * r->view_cap, r->n_slots, r->nwords, r->cap_entries,
                                r->cap_act,
                                (int64_t)1});
    size_t need = sizeof(unsigned long long) * (scan_tiles(biggest) + 1);
    if (r->scan_status[0].bytes >= need) return SPR_OK;
    drop_graph(r);
    for (DevBuf &b : r->scan_status) {
        SPR_TRY(buf_reserve(b, need, s));
        SPR_CUDA_TRY(cudaMemsetAsync(b.p, 0, b.bytes, s));
    }
    return SPR_OK;
}

// Empty the cache.  The first time (and after the slot tables are
// reallocated) every table is cleared; afterwards only the used slots are
// undone, which costs O(slots used) instead of O(blocks).
int reset_cache(spr_renderer *r, cudaStream_t s)
{
    const VolGeom &g = r->vol->g;
    if (!r->cache_init) {
        SPR_CUDA_TRY(cudaMemsetAsync(r->blk_slot.p, 0xFF, sizeof(uint32_t) * g.nblocks, s));
        SPR_CUDA_TRY(cudaMemsetAsync(r->slot_blk.p, 0xFF, sizeof(uint32_t) * r->n_slots, s));
        SPR_CUDA_TRY(cudaMemsetAsync(r->touched.p, 0, r->n_slots, s));
        r->cache_init = true;
    } else {
        cache_clear_used_kernel<<<grid_for(r->n_slots, 256, 8), 256, 0, s>>>(
            r->ps.as<PassState>(), nullptr, r->slot_blk.as<uint32_t>(), r->blk_slot.as<uint32_t>(),
            r->touched.as<uint8_t>(), r->n_slots);
        count_launch();
    }
    // every slot is fresh again; the used-slot lists are empty
    cache_reset_kernel<<<1, 32, 0, s>>>(r->ps.as<PassState>(), nullptr);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    r->cache_dirty = false;
    return SPR_OK;
}

Geo make_geo(const spr_renderer *r)
{
    Geo P;
    P.g = r->vol->g;
    P.fine = r->vol->fine.as<float2>();
    P.coarse = r->vol->coarse.as<float2>();
    P.views = r->camd.as<DevParams>()->views;
    P.W = r->W;
    P.H = r->H;
    P.WH = (int64_t)r->W * r->H;
    P.fstride = r->vol->g.ncoarse;
    P.sstride = (int64_t)r->occ.ns[0] * r->occ.ns[1] * r->occ.ns[2];
    P.occ = r->occ;
    return P;
}

// occupancy bitmaps for the current isovalue (recomputed when it changes)
int update_occupancy(spr_renderer *r, cudaStream_t s)
{
    const VolGeom &g = r->vol->g;
    const int64_t ns = (int64_t)r->occ.ns[0] * r->occ.ns[1] * r->occ.ns[2];
    for (int v = 0; v < r->n_views; ++v) {
        const float iso = r->views[v].iso;
        if (r->occ_iso[v] == iso) continue;
        unsigned long long *fm = r->occ_fine.as<unsigned long long>() + v * g.ncoarse;
        unsigned long long *sm = r->occ_super.as<unsigned long long>() + v * ns;
        int *box = r->occ_box.as<int>() + 8 * v;
        SPR_CUDA_TRY(cudaMemsetAsync(box, 0x7F, 4 * sizeof(int), s));       // lo: 0x7F7F7F7F
        SPR_CUDA_TRY(cudaMemsetAsync(box + 4, 0xFF, 4 * sizeof(int), s));   // hi: -1
        fmask_kernel<<<grid_for(g.ncoarse, 128, 16), 128, 0, s>>>(r->vol->fine.as<float2>(), g, iso, fm, box);
        smask_kernel<<<grid_for(ns, 128, 16), 128, 0, s>>>(fm, g, r->occ, sm);
        count_launch(2);
        SPR_CUDA_TRY(cudaGetLastError());
        r->occ_iso[v] = iso;
    }
    return SPR_OK;
}

// bytes of the parameter block that are copied: the header and view_cap
// views (the start graph's copy node keeps its size while the active count
// changes within the capacity; views past n_views are not read)
inline size_t params_bytes(const spr_renderer *r)
{
    return offsetof(DevParams, views) + sizeof(View) * (size_t)r->view_cap;
}

// Fill the pinned parameter block (after the previous copy out of it ran).
int write_params(spr_renderer *r, uint32_t more, uint32_t reset)
{
    SPR_CUDA_TRY(cudaEventSynchronize(r->ev_upload));
    DevParams &h = *r->h_params;
    h.n_views = (uint32_t)r->n_views;
    for (int v = 0; v < r->n_views; ++v) h.views[v] = r->views[v];
    h.spec_mode = (uint32_t)r->spec_mode;
    h.k_fixed = (uint32_t)r->k_fixed;
    h.k_max = (uint32_t)r->k_max;
    h.npix = (uint32_t)r->npix;
    h.more = more;
    h.reset = reset;
    h.coop_below = r->coop_below;
    h.seg_threads = r->seg_threads;
    return SPR_OK;
}

// camera, isovalue and the speculation configuration to the device (the
// host-driven path; the graph path copies them inside its start graph)
int upload_params(spr_renderer *r, cudaStream_t s)
{
    if (!r->params_dirty) return SPR_OK;
    SPR_TRY(write_params(r, 0u, 0u));
    SPR_CUDA_TRY(cudaMemcpyAsync(r->camd.p, r->h_params, params_bytes(r), cudaMemcpyHostToDevice, s));
    SPR_CUDA_TRY(cudaEventRecord(r->ev_upload, s));
    config_kernel<<<1, 32, 0, s>>>(r->ps.as<PassState>(), r->camd.as<DevParams>());
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    r->params_dirty = false;
    return SPR_OK;
}

// ray generation, device work only (capturable): rays, live list 0, pass state
// In the start graph (dp given) the counters were zeroed by start_kernel,
// ray generation resets the LRU state when asked and after_raygen applies
// the pass limit; eagerly (dp null) the counters are zeroed here.
int enqueue_raygen_body(spr_renderer *r, cudaStream_t s, const DevParams *dp)
{
    uint32_t *ctr = r->ctr.as<uint32_t>();
    if (!dp) SPR_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * C_COUNT, s));
    const int64_t n_tiled = tiled_ray_count(r->W, r->H) * r->view_cap;
    raygen_kernel<<<grid_for(n_tiled, 256, 8), 256, 0, s>>>(
        make_geo(r), r->H, r->state_in.as<uint64_t>(), r->status.as<uint8_t>(), r->keys.as<uint64_t>(),
        r->fb_depth.as<float>(), r->fb_rgba.as<uint32_t>(), r->fb_block.as<uint32_t>(), r->fb_cell.as<uint64_t>(),
        r->fb_final.as<int32_t>(), r->lbits.as<uint32_t>(), n_tiled, r->ps.as<PassState>(),
        dp ? &dp->reset : nullptr, dp ? &dp->n_views : nullptr, (uint32_t)r->n_views);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    SPR_TRY(run_compact(r->scan_status[0], r->scan_ticket[0], ctr + C_SCANFLAGS, n_tiled, nullptr,
                        BitCount{r->lbits.as<uint32_t>(), nullptr},
                        EnterEmit{r->live[0].as<uint32_t>(), r->W, r->H, (int64_t)r->W * r->H}, ctr + C_NLIVE,
                        s));
    after_raygen_kernel<<<1, 32, 0, s>>>(r->ps.as<PassState>(), ctr, r->d_hps, dp ? &dp->more : nullptr);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    return SPR_OK;
}

// Each attempt clears the bitmaps after their last reader.  A render that
// stopped on a device error clears them here before the next one.
int clear_bits_if_dirty(spr_renderer *r, cudaStream_t s)
{
    if (!r->bits_dirty) return SPR_OK;
    SPR_CUDA_TRY(cudaMemsetAsync(r->vis_bits.p, 0, sizeof(uint32_t) * r->nwords, s));
    SPR_CUDA_TRY(cudaMemsetAsync(r->act_bits.p, 0, sizeof(uint32_t) * r->nwords, s));
    r->bits_dirty = false;
    return SPR_OK;
}

// ray generation (no host synchronisation)
int enqueue_raygen(spr_renderer *r, cudaStream_t s)
{
    SPR_TRY(update_occupancy(r, s));
    SPR_TRY(clear_bits_if_dirty(r, s));
    SPR_TRY(enqueue_raygen_body(r, s, nullptr));
    r->need_raygen = false;
    r->pass = 0;
    return SPR_OK;
}

// start of a call that continues a render: LRU reset if asked, pass limit
__global__ void limit_kernel(PassState *ps, const DevParams *p)
{
    if (threadIdx.x != 0) return;
    if (p->reset) lru_reset(ps);
    ps->max_passes = ps->pass + p->more;
    ps->run = (ps->n_live > 0 && p->more > 0) ? 1u : 0u;
}

// allow `more` passes (*more_dev when given) from the current one
__global__ void set_limit_kernel(PassState *ps, uint32_t more, const uint32_t *more_dev)
{
    if (threadIdx.x != 0) return;
    if (more_dev) more = *more_dev;
    ps->max_passes = ps->pass + more;
    ps->run = (ps->n_live > 0 && more > 0) ? 1u : 0u;
}

// an event record that also works inside stream capture (as an event node)
inline cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing)
{
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// One attempt of a pass, entirely on the device.  Capturable: no host
// synchronisation and no host-side scalars that change between passes.
// With events, records ev[0..6] around the stages and runs them in order;
// without, the grouping and cache stages run as concurrent branches:
//
//   main:  begin, traverse --+-- visible scan ---(active)--- entry counts,
//                            |                               offsets, scatter --(decode)-- intersect, resolve --(lru)-- end
//   aux 0:                   +-- active scan -- lookup -- victims -- assign --+-- decode
//   aux 1:                                                                   +-- LRU order scan
//
// The bitmaps are cleared right after their last reader, ready for the next
// attempt.
int launch_policy(spr_renderer *r, cudaStream_t s)
{
    // persistent CTAs: at most four per SM (256 of the 512 TMEM columns,
    // 134 KB of shared memory), never more than there are tiles
    const int64_t tiles = (r->npix_cap + mlp::kRows - 1) / mlp::kRows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 4 * device_sm_count()));
    policy_kernel<<<grid, mlp::kRows, 0, s>>>(make_geo(r), r->live[0].as<uint32_t>(), r->live[1].as<uint32_t>(),
                                              r->ps.as<PassState>(), r->state_in.as<uint64_t>(),
                                              r->policy.as<float>(), r->kray.as<uint32_t>(), r->ctr.as<uint32_t>());
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    return SPR_OK;
}

Trace make_trace(spr_renderer *r)
{
    Trace T{};
    if (!r->tracing) return T;
    T.feat = r->tr_feat;
    T.ray = r->tr_ray;
    T.cons = r->tr_cons;
    T.count = r->tr_count.as<uint32_t>();
    T.cap = r->tr_cap;
    T.mod = r->tr_mod;
    T.taken = r->tr_taken.as<uint32_t>();
    T.need = r->tr_need.as<uint32_t>();
    return T;
}

// Whether a pass can ever walk one ray per warp: the warp walks take passes
// of fewer than coop_below rays that the segmented walk leaves alone (fewer
// than two lanes per ray), which cannot happen when seg_threads >= 2 *
// coop_below; then their kernels are not launched (an idle launch of 2,432
// CTAs costs about 5 us per pass).
bool coop_walks_possible(const spr_renderer *r)
{
    return r->coop_below > 0 && (r->seg_threads == 0 || (uint64_t)r->seg_threads < 2ull * r->coop_below);
}

// After the assignment (which marks the victims and the fresh slots it
// hands out): the next pass's LRU list, the untouched used slots in order,
// then the touched ones in slot order.
int enqueue_lru_order(spr_renderer *r, const LruPair &lp, uint32_t *flags, cudaStream_t s)
{
    uint32_t *ctr = r->ctr.as<uint32_t>();
    PassState *ps = r->ps.as<PassState>();
    SPR_TRY(run_compact(r->scan_status[2], r->scan_ticket[2], flags, r->n_slots, &ps->n_used,
                        KeepCount{lp, r->touched.as<uint8_t>(), ctr + C_OVERFLOW}, KeepEmit{lp}, ctr + C_NUNTOUCHED,
                        s));
    SPR_TRY(run_compact(r->scan_status[2], r->scan_ticket[2], flags, r->n_slots, &ps->fresh_hi,
                        TouchedCount{r->touched.as<uint8_t>(), ctr + C_OVERFLOW},
                        TouchedEmit{r->touched.as<uint8_t>(), ctr, lp}, nullptr, s));
    return SPR_OK;
}

int enqueue_attempt(spr_renderer *r, cudaStream_t s, bool events, cudaGraphConditionalHandle h, int use_h,
                    bool capturing = false)
{
    const VolGeom &g = r->vol->g;
    uint32_t *ctr = r->ctr.as<uint32_t>();
    uint32_t *flags = ctr + C_SCANFLAGS;
    PassState *ps = r->ps.as<PassState>();
    uint32_t *live0 = r->live[0].as<uint32_t>(), *live1 = r->live[1].as<uint32_t>();
    const int64_t cap = r->cap_entries;
    const bool fork = !events;
    cudaStream_t sa = fork ? r->aux[0] : s;   // cache branch
    cudaStream_t sl = fork ? r->aux[1] : s;   // LRU order branch
    cudaEvent_t ev_trav = r->jev[0], ev_act = r->jev[1], ev_dec = r->jev[3], ev_lru = r->jev[4];
    int64_t k0 = r->launches;
    if (events) SPR_CUDA_TRY(record(r->ev[0], s, capturing));
    begin_pass_kernel<<<1, 32, 0, s>>>(ps, ctr);
    count_launch();

    // training traces: record this pass's samples before the walk moves on
    const Trace T = make_trace(r);
    if (T.taken) {
        trace_kernel<<<grid_for(r->npix_cap, 128, 8), 128, 0, s>>>(make_geo(r), live0, live1, ps,
                                                                   r->state_in.as<uint64_t>(), T);
        count_launch();
    }

    // per-ray speculation: each live ray's count, then their offsets
    Spec S{nullptr, nullptr, nullptr};
    if (per_ray_mode(r->spec_mode)) {
        S = Spec{r->kray.as<uint32_t>(), r->koff.as<uint32_t>(), r->eray.as<uint32_t>()};
        if (r->spec_mode == SPR_SPEC_LEARNED)
            SPR_TRY(launch_policy(r, s));
        else {
            hashed_k_kernel<<<grid_for(r->npix_cap, 256, 8), 256, 0, s>>>(live0, live1, ps, r->kray.as<uint32_t>());
            count_launch();
        }
        SPR_TRY(run_compact(r->scan_status[0], r->scan_ticket[0], flags, r->npix_cap, &ps->nproc,
                            ArrayCount{r->kray.as<uint32_t>(), nullptr}, ArrayEmit{r->koff.as<uint32_t>()},
                            ctr + C_KTOT, s));
    }

    // (a) traversal with speculation, marking visible and active blocks
    traverse_kernel<<<grid_for(r->npix_cap, 128, 16), 128, 0, s>>>(
        make_geo(r), live0, live1, ps, r->state_in.as<uint64_t>(), r->state_out.as<uint64_t>(),
        r->rbid.as<uint32_t>(), r->vis_bits.as<uint32_t>(), r->act_bits.as<uint32_t>(), ctr, S);
    count_launch();
    if (coop_walks_possible(r)) {
        traverse_coop_kernel<32><<<device_sm_count() * 16, 128, 0, s>>>(
            make_geo(r), live0, live1, ps, r->state_in.as<uint64_t>(), r->state_out.as<uint64_t>(),
            r->rbid.as<uint32_t>(), r->vis_bits.as<uint32_t>(), r->act_bits.as<uint32_t>(), ctr, S);
        count_launch();
        traverse_coop_kernel<16><<<device_sm_count() * 16, 128, 0, s>>>(
            make_geo(r), live0, live1, ps, r->state_in.as<uint64_t>(), r->state_out.as<uint64_t>(),
            r->rbid.as<uint32_t>(), r->vis_bits.as<uint32_t>(), r->act_bits.as<uint32_t>(), ctr, S);
        count_launch();
    }
    if (r->seg_threads) {
        traverse_seg_kernel<<<device_sm_count() * 16, kSegThreads, 0, s>>>(
            make_geo(r), live0, live1, ps, r->state_in.as<uint64_t>(), r->state_out.as<uint64_t>(),
            r->rbid.as<uint32_t>(), r->vis_bits.as<uint32_t>(), r->act_bits.as<uint32_t>(), ctr, S);
        count_launch();
    }
    SPR_CUDA_TRY(cudaGetLastError());
    if (events) SPR_CUDA_TRY(record(r->ev[1], s, capturing));
    if (fork) {
        SPR_CUDA_TRY(cudaEventRecord(ev_trav, s));
        SPR_CUDA_TRY(cudaStreamWaitEvent(sa, ev_trav, 0));
    }

    // (b) compact the marks; group the entries by visible block.  The active
    // scan (cache branch) decides whether the pass overflows the cache and
    // leaves the active bitmap zero for the next attempt.
    uint32_t *tsum = r->bits_tsum.as<uint32_t>();
    SPR_TRY(run_bits_compact(r->act_bits.as<uint32_t>(), r->nwords, tsum,
                             BitsEmit{r->act_bits.as<uint32_t>(), nullptr, r->iact.as<uint32_t>(), nullptr},
                             ctr + C_NACT, sa, ctr + C_OVERFLOW, (uint32_t)r->n_slots, true));
    if (fork) SPR_CUDA_TRY(cudaEventRecord(ev_act, sa));
    SPR_TRY(run_bits_compact(r->vis_bits.as<uint32_t>(), r->nwords, tsum + bits_tiles(r->nwords),
                             BitsEmit{r->vis_bits.as<uint32_t>(), r->vis_wpre.as<uint32_t>(), r->ivis.as<uint32_t>(),
                                      r->nbrays.as<uint32_t>()},
                             ctr + C_NVIS, s));
    if (fork) SPR_CUDA_TRY(cudaStreamWaitEvent(s, ev_act, 0));
    count_entries_kernel<<<grid_for(cap, 256, 4), 256, 0, s>>>(
        ps, r->rbid.as<uint32_t>(), r->vis_bits.as<uint32_t>(), r->vis_wpre.as<uint32_t>(),
        r->nbrays.as<uint32_t>(), r->erank.as<uint32_t>(), ctr, S);
    count_launch();
    SPR_TRY(run_compact(r->scan_status[0], r->scan_ticket[0], flags, cap, ctr + C_NVIS,
                        ArrayCount{r->nbrays.as<uint32_t>(), ctr + C_OVERFLOW},
                        ArrayEmit{r->obrays.as<uint32_t>()}, ctr + C_NENT, s));
    scatter_entries_kernel<<<grid_for(cap, 256, 4), 256, 0, s>>>(
        ps, r->rbid.as<uint32_t>(), r->vis_bits.as<uint32_t>(), r->vis_wpre.as<uint32_t>(),
        r->obrays.as<uint32_t>(), r->erank.as<uint32_t>(), r->E.as<uint32_t>(), ctr, S);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    SPR_CUDA_TRY(cudaMemsetAsync(r->vis_bits.p, 0, sizeof(uint32_t) * r->nwords, s));
    if (events) SPR_CUDA_TRY(record(r->ev[2], s, capturing));

    // (c) cache: look up, pick least recently used victims, assign
    LruPair lp{r->lru[0].as<uint32_t>(), r->lru[1].as<uint32_t>(), ps};
    SPR_TRY(run_compact(r->scan_status[1], r->scan_ticket[1], flags, r->cap_act, ctr + C_NACT,
                        LookupCount{r->iact.as<uint32_t>(), r->blk_slot.as<uint32_t>(), ctr + C_OVERFLOW},
                        LookupEmit{r->iact.as<uint32_t>(), r->blk_slot.as<uint32_t>(), r->touched.as<uint8_t>(),
                                   r->miss.as<uint32_t>()},
                        ctr + C_NMISS, sa));
    SPR_TRY(run_compact(r->scan_status[1], r->scan_ticket[1], flags, r->n_slots, &ps->n_used,
                        VictimCount{lp, r->touched.as<uint8_t>(), ctr, (uint32_t)r->n_slots},
                        VictimEmit{lp, ctr, r->victim.as<uint32_t>(), (uint32_t)r->n_slots}, nullptr, sa));
    if (events) SPR_CUDA_TRY(record(r->ev[3], s, capturing));

    // (d) decode the misses into their slots, the decoder handing out the
    // slots (fresh ones first, then the victims) as it reads the misses
    SPR_TRY(launch_decode_sorted(r->vol->comp.as<uint8_t>(), g.nblocks, g.rate, r->vol->planes.as<uint8_t>(),
                                 r->miss.as<uint32_t>(),
                                 AssignSlot{r->victim.as<uint32_t>(), r->blk_slot.as<uint32_t>(),
                                            r->slot_blk.as<uint32_t>(), r->touched.as<uint8_t>(), ctr, ps,
                                            (uint32_t)r->n_slots},
                                 r->cap_act, ctr + C_NMISS, ctr + C_OVERFLOW, r->cache.as<float>(), ctr + C_BAD, sa));
    count_launch();
    if (events) SPR_CUDA_TRY(record(r->ev[4], s, capturing));
    if (fork) {
        SPR_CUDA_TRY(cudaEventRecord(ev_dec, sa));
        SPR_CUDA_TRY(cudaStreamWaitEvent(s, ev_dec, 0));
        SPR_CUDA_TRY(cudaStreamWaitEvent(sl, ev_dec, 0));
        SPR_TRY(enqueue_lru_order(r, lp, flags, sl));   // beside the intersection
    }

    // (e) intersect the entries, block by block
    RT R{make_geo(r), r->cache.as<float>(), r->blk_slot.as<uint32_t>()};
    if (r->isect_staged)
        intersect_staged_kernel<<<device_sm_count() * 4, 32 * kStageWarps, 0, s>>>(
            R, r->E.as<uint32_t>(), r->rbid.as<uint32_t>(), live0, live1, ps, r->keys.as<unsigned long long>(), ctr,
            S);
    else
        intersect_kernel<<<r->grid_isect, 128, 0, s>>>(R, r->E.as<uint32_t>(), r->rbid.as<uint32_t>(), live0, live1,
                                                       ps, r->keys.as<unsigned long long>(), ctr, S);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    if (events) SPR_CUDA_TRY(record(r->ev[5], s, capturing));

    // (f) resolve hits and exits, compact the live rays in order, end the pass
    resolve_kernel<<<grid_for(r->npix_cap, 256, 8), 256, 0, s>>>(
        live0, live1, ps, g.dims[0], g.dims[1], g, r->keys.as<unsigned long long>(), r->rbid.as<uint32_t>(),
        r->state_in.as<uint64_t>(), r->state_out.as<uint64_t>(), r->status.as<uint8_t>(), r->fb_depth.as<float>(),
        r->fb_rgba.as<uint32_t>(), r->fb_block.as<uint32_t>(), r->fb_cell.as<uint64_t>(), r->fb_final.as<int32_t>(),
        r->lbits.as<uint32_t>(), ctr, S, T);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    SPR_TRY(run_compact(r->scan_status[0], r->scan_ticket[0], flags, r->npix_cap, &ps->n_live,
                        BitCount{r->lbits.as<uint32_t>(), ctr + C_OVERFLOW}, LiveEmit{live0, live1, ps},
                        ctr + C_NLIVE, s));
    if (fork) {   // the LRU order must be complete before the pass ends
        SPR_CUDA_TRY(cudaEventRecord(ev_lru, sl));
        SPR_CUDA_TRY(cudaStreamWaitEvent(s, ev_lru, 0));
    } else {
        SPR_TRY(enqueue_lru_order(r, lp, flags, s));
    }
    end_pass_kernel<<<1, 32, 0, s>>>(ps, ctr, r->d_recs, (uint32_t)spr_renderer::kRecCap, r->d_hps, h, use_h);
    count_launch();
    SPR_CUDA_TRY(cudaGetLastError());
    if (events) SPR_CUDA_TRY(record(r->ev[6], s, capturing));
    r->graph_kernels = (int)(r->launches - k0);
    return SPR_OK;
}

int check_ready(spr_renderer *r)
{
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    const uint64_t all = r->n_views == 64 ? ~0ull : ((1ull << r->n_views) - 1);
    if ((r->cam_set & all) != all) return set_error(SPR_ERR_INVALID_ARG, "a view has no camera");
    if (r->n_slots < 8) return set_error(SPR_ERR_CACHE_TOO_SMALL, "cache budget below 8 slots");
    return SPR_OK;
}

int prepare(spr_renderer *r, cudaStream_t s)
{
    SPR_TRY(check_ready(r));
    SPR_TRY(ensure_entry_buffers(r, s));
    SPR_TRY(ensure_scan_scratch(r, s));
    SPR_TRY(upload_params(r, s));
    if (r->cache_dirty) SPR_TRY(reset_cache(r, s));
    return SPR_OK;
}

int read_state(spr_renderer *r, cudaStream_t s)
{
    SPR_CUDA_TRY(cudaStreamSynchronize(s));   // h_ps is written by the last pass kernel
    const PassState &h = *r->h_ps;
    r->n_live = h.n_live;
    r->n_enter = h.n_enter;
    r->pass = (int)h.pass;
    if (h.error) r->bits_dirty = true;
    if (h.error & 1u) return set_error(SPR_ERR_DEVICE_TIMEOUT, "a decoupled look-back wait timed out");
    if (h.error & 2u) return set_error(SPR_ERR_DEVICE_ERROR, "a kernel flagged an out-of-range block id");
    if (h.error & 4u) return set_error(SPR_ERR_DEVICE_ERROR, "a traversal exceeded its step bound");
    if (h.error & 16u) return set_error(SPR_ERR_DEVICE_TIMEOUT, "a tensor-core wait of the speculation policy timed out");
    return SPR_OK;
}

int build_prof_graph(spr_renderer *r);

// one pass driven from the host (used by spr_render_pass and for per-stage
// timing): attempts until the pass completes
int do_pass(spr_renderer *r, cudaStream_t s, spr_pass_stats *out)
{
    SPR_TRY(prepare(r, s));
    struct Scope {
        Scope(int64_t *p) { g_launch_counter = p; }
        ~Scope() { g_launch_counter = nullptr; }
    } scope(&r->launches);
    const bool prof = r->profiling;
    if (r->need_raygen) {
        r->launches = 0;
        if (prof) SPR_CUDA_TRY(cudaEventRecord(r->ev[7], s));
        SPR_TRY(enqueue_raygen(r, s));
        if (prof) {
            SPR_CUDA_TRY(cudaEventRecord(r->ev[0], s));
            SPR_CUDA_TRY(cudaEventSynchronize(r->ev[0]));
            cudaEventElapsedTime(&r->ms_raygen, r->ev[7], r->ev[0]);
        }
    }
    SPR_TRY(read_state(r, s));
    spr_pass_stats st;
    memset(&st, 0, sizeof st);
    st.pass = r->pass;
    if (r->n_live == 0) {
        if (out) *out = st;
        return SPR_OK;
    }
    set_limit_kernel<<<1, 32, 0, s>>>(r->ps.as<PassState>(), 1u, nullptr);
    count_launch();
    float stage_ms[6] = {0, 0, 0, 0, 0, 0};
    const int before = r->pass;
    if (prof) SPR_TRY(build_prof_graph(r));
    for (int attempt = 0; attempt < 64 && r->pass == before; ++attempt) {
        if (prof) {
            SPR_CUDA_TRY(cudaGraphLaunch(r->gprof, s));
            r->launches += r->graph_kernels;
        } else {
            SPR_TRY(enqueue_attempt(r, s, false, 0, 0));
        }
        SPR_TRY(read_state(r, s));
        if (prof)
            for (int k = 0; k < 6; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, r->ev[k], r->ev[k + 1]);
                stage_ms[k] += ms;
            }
    }
    if (r->pass == before) return set_error(SPR_ERR_DEVICE_ERROR, "a pass did not fit the cache after 64 attempts");
    if (before < spr_renderer::kRecCap) {
        st = r->h_recs[before];   // written by the pass's last kernel; the stream was synchronised
    } else {
        st.pass = before + 1;   // past the record buffer: counts only in the render totals
    }
    float tot = 0.f;
    for (int i = 0; i < 6; ++i) {
        st.ms_stage[i] = stage_ms[i];
        tot += stage_ms[i];
    }
    st.ms = tot;
    if (out) *out = st;
    return SPR_OK;
}

// One attempt captured with event nodes between its stages, so that stage
// times are device times, free of host launch gaps.
int build_prof_graph(spr_renderer *r)
{
    if (r->gprof) return SPR_OK;
    if (!r->cap_stream) SPR_CUDA_TRY(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
    SPR_CUDA_TRY(cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal));
    int64_t saved = r->launches;
    int rc = enqueue_attempt(r, r->cap_stream, true, 0, 0, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(r->cap_stream, &g);
    r->launches = saved;
    if (rc != SPR_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != SPR_OK ? rc : set_error(SPR_ERR_CUDA, "profiling capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&r->gprof, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        r->gprof = nullptr;
        return set_error(SPR_ERR_CUDA, "profiling graph: %s", cudaGetErrorString(e));
    }
    return SPR_OK;
}

// Buffers sized by the rays of all views: per-ray state, live lists, keys,
// framebuffer, the enter/alive bitmap and the brick masks (one set per view).
// Frees the previous ones first.
int alloc_view_buffers(spr_renderer *r)
{
    cudaStream_t s = nullptr;
    DevBuf *bufs[] = {&r->state_in, &r->state_out, &r->status, &r->live[0], &r->live[1], &r->keys,
                      &r->fb_depth, &r->fb_rgba, &r->fb_block, &r->fb_cell, &r->fb_final, &r->lbits,
                      &r->occ_fine, &r->occ_super, &r->occ_box};
    for (DevBuf *b : bufs) buf_free(*b, s);
    const int64_t np = r->npix_cap;
    const int64_t ns = (int64_t)r->occ.ns[0] * r->occ.ns[1] * r->occ.ns[2];
    int rc;
    if ((rc = buf_alloc(r->state_in, 8 * np, s)) || (rc = buf_alloc(r->state_out, 8 * np, s)) ||
        (rc = buf_alloc(r->status, np, s)) || (rc = buf_alloc(r->live[0], 4 * np, s)) ||
        (rc = buf_alloc(r->live[1], 4 * np, s)) || (rc = buf_alloc(r->keys, 8 * np, s)) ||
        (rc = buf_alloc(r->fb_depth, 4 * np, s)) || (rc = buf_alloc(r->fb_rgba, 4 * np, s)) ||
        (rc = buf_alloc(r->fb_block, 4 * np, s)) || (rc = buf_alloc(r->fb_cell, 8 * np, s)) ||
        (rc = buf_alloc(r->fb_final, 4 * np, s)) ||
        (rc = buf_alloc(r->lbits, 4 * (tiled_ray_count(r->W, r->H) * r->view_cap / 32 + 1), s)) ||
        (rc = buf_alloc(r->occ_fine, 8 * r->vol->g.ncoarse * r->view_cap, s)) ||
        (rc = buf_alloc(r->occ_super, 8 * ns * r->view_cap, s)) ||
        (rc = buf_alloc(r->occ_box, 32 * r->view_cap, s)))
        return rc;
    r->occ.fmask = r->occ_fine.as<unsigned long long>();
    r->occ.smask = r->occ_super.as<unsigned long long>();
    r->occ.box = r->occ_box.as<int>();
    for (int v = 0; v < kMaxViews; ++v) r->occ_iso[v] = NAN;
    return SPR_OK;
}

// The start of a render as one graph: copy the parameter block, apply the
// speculation settings, empty the cache if asked, generate rays (with_raygen)
// and set the pass limit.  Kernels in it: 4 with ray generation, else 2.
// The start of a render captured into a new graph g (not instantiated).
int capture_start_graph(spr_renderer *r, bool with_raygen, cudaGraph_t *out)
{
    *out = nullptr;
    if (!r->cap_stream) SPR_CUDA_TRY(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = r->cap_stream;
    DevParams *dp = r->camd.as<DevParams>();
    PassState *ps = r->ps.as<PassState>();
    SPR_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int64_t saved = r->launches;
    int rc = SPR_OK;
    cudaError_t e = cudaMemcpyAsync(dp, r->h_params, params_bytes(r), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) {
        start_kernel<<<grid_for(r->n_slots, 256, 8), 256, 0, cs>>>(ps, dp, r->ctr.as<uint32_t>(),
                                                                  r->slot_blk.as<uint32_t>(),
                                                                  r->blk_slot.as<uint32_t>(),
                                                                  r->touched.as<uint8_t>(), r->n_slots);
        if (with_raygen) rc = enqueue_raygen_body(r, cs, dp);
        else limit_kernel<<<1, 32, 0, cs>>>(ps, dp);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    r->launches = saved;
    if (e != cudaSuccess || e2 != cudaSuccess || rc != SPR_OK) {
        if (g) cudaGraphDestroy(g);
        if (rc != SPR_OK) return rc;
        return set_error(SPR_ERR_CUDA, "start capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    *out = g;
    return SPR_OK;
}

int build_start_graph(spr_renderer *r, bool with_raygen)
{
    cudaGraphExec_t &ge = with_raygen ? r->gstart : r->glimit;
    if (ge) return SPR_OK;
    cudaGraph_t g = nullptr;
    SPR_TRY(capture_start_graph(r, with_raygen, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ge = nullptr;
        return set_error(SPR_ERR_CUDA, "start graph: %s", cudaGetErrorString(e));
    }
    return SPR_OK;
}

// Capture the pass loop once: a conditional while node whose body is one
// attempt; end_pass_kernel sets the condition.
int build_graph(spr_renderer *r)
{
    if (r->gexec) return SPR_OK;
    if (!r->cap_stream) SPR_CUDA_TRY(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    SPR_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_error(SPR_ERR_CUDA, "conditional graph node: %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(r->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    int rc = SPR_OK;
    int64_t saved = r->launches;
    if (e == cudaSuccess) rc = enqueue_attempt(r, r->cap_stream, false, h, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(r->cap_stream, &captured);
    r->launches = saved;
    if (e != cudaSuccess || e2 != cudaSuccess || rc != SPR_OK) {
        cudaGraphDestroy(g);
        if (rc != SPR_OK) return rc;
        return set_error(SPR_ERR_CUDA, "pass capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&r->gexec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        r->gexec = nullptr;
        return set_error(SPR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    r->graph = g;
    return SPR_OK;
}

}  // namespace

// settings and synchronous renders wait until a submitted render is collected
static int check_idle(const spr_renderer *r)
{
    if (r->busy) return set_error(SPR_ERR_INVALID_ARG, "a submitted render has not been collected");
    return SPR_OK;
}

extern "C" int spr_create_renderer(spr_volume *vol, int width, int height, spr_renderer **out)
{
    clear_error();
    if (!vol || !out || width < 1 || height < 1) return set_error(SPR_ERR_INVALID_ARG, "bad renderer arguments");
    *out = nullptr;
    if ((int64_t)width * height > (int64_t)1 << 28) return set_error(SPR_ERR_INVALID_ARG, "image too large");
    // the decoder's shared-memory attribute, set here, outside any capture
    SPR_TRY(decode_sorted_prepare<AssignSlot>(nullptr));
    spr_renderer *r = new (std::nothrow) spr_renderer();
    if (!r) return set_error(SPR_ERR_OUT_OF_MEMORY, "host allocation failed");
    r->vol = vol;
    r->W = width;
    r->H = height;
    r->npix = (int64_t)width * height;
    r->npix_cap = r->npix;
    r->nwords = (vol->g.nblocks + 31) / 32;
    r->n_slots = (int64_t)(256u << 20) / 256;
    cudaStream_t s = nullptr;
    int rc = SPR_OK;
    for (int v = 0; v < kMaxViews; ++v) {
        r->views[v].iso = r->iso;
        r->occ_iso[v] = NAN;
    }
    if ((rc = buf_alloc(r->vis_bits, 4 * r->nwords, s)) ||
        (rc = buf_alloc(r->act_bits, 4 * r->nwords, s)) || (rc = buf_alloc(r->vis_wpre, 4 * r->nwords, s)) ||
        (rc = buf_alloc(r->bits_tsum, 8 * bits_tiles(r->nwords), s)) ||
        (rc = buf_alloc(r->blk_slot, 4 * vol->g.nblocks, s)) || (rc = buf_alloc(r->scan_ticket[0], 64, s)) ||
        (rc = buf_alloc(r->scan_ticket[1], 64, s)) || (rc = buf_alloc(r->scan_ticket[2], 64, s)) ||
        (rc = buf_alloc(r->ctr, sizeof(uint32_t) * C_COUNT, s)) ||
        (rc = buf_alloc(r->ps, sizeof(PassState), s)) ||
        (rc = buf_alloc(r->camd, sizeof(DevParams) + 16, s))) {
        free_all(r);
        delete r;
        return rc;
    }
    if (cudaMemset(r->ps.p, 0, sizeof(PassState)) != cudaSuccess ||
        cudaMemset(r->scan_ticket[0].p, 0, 64) != cudaSuccess || cudaMemset(r->scan_ticket[1].p, 0, 64) != cudaSuccess ||
        cudaMemset(r->scan_ticket[2].p, 0, 64) != cudaSuccess ||
        cudaMemset(r->vis_bits.p, 0, 4 * r->nwords) != cudaSuccess ||
        cudaMemset(r->act_bits.p, 0, 4 * r->nwords) != cudaSuccess ||
        cudaMallocHost((void **)&r->h_ctr, sizeof(uint32_t) * C_COUNT) != cudaSuccess ||
        cudaHostAlloc((void **)&r->h_ps, sizeof(PassState), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&r->d_hps, r->h_ps, 0) != cudaSuccess ||
        cudaHostAlloc((void **)&r->h_recs, sizeof(spr_pass_stats) * spr_renderer::kRecCap, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer((void **)&r->d_recs, r->h_recs, 0) != cudaSuccess ||
        cudaMallocHost((void **)&r->h_params, sizeof(DevParams)) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_upload, cudaEventDisableTiming) != cudaSuccess) {
        free_all(r);
        delete r;
        return set_error(SPR_ERR_OUT_OF_MEMORY, "pinned host allocation failed");
    }
    memset(r->h_ps, 0, sizeof(PassState));
    memset(r->h_recs, 0, sizeof(spr_pass_stats) * spr_renderer::kRecCap);
    for (auto &e : r->ev) cudaEventCreate(&e);
    for (auto &e : r->jev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    for (auto &a : r->aux) cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
    // one wave of the work-queue kernel
    {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, intersect_kernel, 128, 0) != cudaSuccess || nb < 1)
            nb = 1;
        r->grid_isect = nb * device_sm_count();
    }
    for (int a = 0; a < 3; ++a) {
        r->occ.ns[a] = (vol->g.nc[a] + 3) / 4;
        r->occ.ts[a] = (vol->g.tc[a] + 3) / 4;
    }
    if ((rc = alloc_view_buffers(r))) {
        free_all(r);
        delete r;
        return rc;
    }
    int64_t slots = r->n_slots;
    r->n_slots = 0;
    if ((rc = spr_set_cache_budget(r, (size_t)slots * 256))) {
        free_all(r);
        delete r;
        return rc;
    }
    *out = r;
    return SPR_OK;
}

extern "C" int spr_destroy_renderer(spr_renderer *r)
{
    clear_error();
    if (!r) return SPR_OK;
    free_all(r);
    delete r;
    return SPR_OK;
}

static bool basis_ok(float x)
{
    float a = fabsf(x);
    return std::isfinite(x) && (a == 0.f || (a >= 0x1p-40f && a <= 0x1p40f));
}

static int check_camera(const float eye[3], const float p00[3], const float du[3], const float dv[3])
{
    if (!eye || !p00 || !du || !dv) return set_error(SPR_ERR_INVALID_ARG, "NULL camera argument");
    for (int a = 0; a < 3; ++a) {
        double e = eye[a];
        if (!std::isfinite(eye[a]) || std::fabs(e) >= 16384.0 || e * 256.0 != std::floor(e * 256.0))
            return set_error(SPR_ERR_INVALID_ARG,
                             "eye[%d] = %.9g must be a multiple of 1/256 below 16384 in magnitude", a, e);
        if (!basis_ok(p00[a]) || !basis_ok(du[a]) || !basis_ok(dv[a]))
            return set_error(SPR_ERR_INVALID_ARG, "camera basis component %d outside {0} or [2^-40, 2^40]", a);
    }
    return SPR_OK;
}

extern "C" int spr_set_view_count(spr_renderer *r, int n_views)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    if (n_views < 1 || n_views > kMaxViews)
        return set_error(SPR_ERR_INVALID_ARG, "n_views = %d outside [1, %d]", n_views, kMaxViews);
    const int64_t np = (int64_t)r->W * r->H * n_views;
    if (np > (int64_t)1 << 28) return set_error(SPR_ERR_INVALID_ARG, "views x width x height above 2^28 rays");
    if (r->spec_mode == SPR_SPEC_FIXED && np * r->k_fixed > 0x7FFFFFFFll)
        return set_error(SPR_ERR_INVALID_ARG, "views x width x height x k exceeds 2^31 entries");
    if (n_views == r->n_views) return SPR_OK;
    r->need_raygen = true;
    r->params_dirty = true;
    if (n_views <= r->view_cap) {
        // within the allocated views: buffers and captured graphs stay
        r->n_views = n_views;
        r->npix = np;
        return SPR_OK;
    }
    cudaDeviceSynchronize();
    drop_graph(r);
    r->n_views = r->view_cap = n_views;
    r->npix = r->npix_cap = np;
    return alloc_view_buffers(r);
}

extern "C" int spr_set_view(spr_renderer *r, int view, const float eye[3], const float p00[3], const float du[3],
                            const float dv[3], float iso)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    if (view < 0 || view >= r->n_views)
        return set_error(SPR_ERR_INVALID_ARG, "view %d outside [0, %d)", view, r->n_views);
    if (!std::isfinite(iso)) return set_error(SPR_ERR_INVALID_ARG, "bad isovalue");
    SPR_TRY(check_camera(eye, p00, du, dv));
    for (int a = 0; a < 3; ++a) {
        r->views[view].cam.eye[a] = eye[a];
        r->views[view].cam.p00[a] = p00[a];
        r->views[view].cam.du[a] = du[a];
        r->views[view].cam.dv[a] = dv[a];
    }
    r->views[view].iso = iso;
    r->cam_set |= 1ull << view;
    r->need_raygen = true;
    r->params_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_camera(spr_renderer *r, const float eye[3], const float p00[3], const float du[3],
                              const float dv[3])
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    SPR_TRY(check_camera(eye, p00, du, dv));
    for (int a = 0; a < 3; ++a) {
        r->views[0].cam.eye[a] = eye[a];
        r->views[0].cam.p00[a] = p00[a];
        r->views[0].cam.du[a] = du[a];
        r->views[0].cam.dv[a] = dv[a];
    }
    r->cam_set |= 1ull;
    r->need_raygen = true;
    r->params_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_isovalue(spr_renderer *r, float iso)
{
    clear_error();
    if (!r || !std::isfinite(iso)) return set_error(SPR_ERR_INVALID_ARG, "bad isovalue");
    SPR_TRY(check_idle(r));
    r->iso = iso;
    for (int v = 0; v < kMaxViews; ++v) r->views[v].iso = iso;
    r->need_raygen = true;
    r->params_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_cache_budget(spr_renderer *r, size_t bytes)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    int64_t slots = (int64_t)(bytes / 256);
    if (slots < 8) return set_error(SPR_ERR_CACHE_TOO_SMALL, "cache budget of %zu bytes is below 8 slots", bytes);
    if (slots > 0x7FFFFFFFll) return set_error(SPR_ERR_INVALID_ARG, "cache budget too large");
    cudaStream_t s = nullptr;
    cudaDeviceSynchronize();
    drop_graph(r);
    buf_free(r->cache, s);
    buf_free(r->slot_blk, s);
    buf_free(r->lru[0], s);
    buf_free(r->lru[1], s);
    buf_free(r->touched, s);
    r->n_slots = 0;
    int rc;
    if ((rc = buf_alloc(r->cache, (size_t)slots * 256, s)) || (rc = buf_alloc(r->slot_blk, 4 * slots, s)) ||
        (rc = buf_alloc(r->lru[0], 4 * slots, s)) || (rc = buf_alloc(r->lru[1], 4 * slots, s)) ||
        (rc = buf_alloc(r->touched, (size_t)slots, s)))
        return rc;
    r->n_slots = slots;
    r->cache_dirty = true;
    r->cache_init = false;
    r->need_raygen = true;
    return SPR_OK;
}

extern "C" int spr_set_speculation(spr_renderer *r, int mode, int k, int k_max)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    if (mode == SPR_SPEC_FIXED) {
        if (k < 1 || k > SPR_K_LIMIT) return set_error(SPR_ERR_INVALID_ARG, "k = %d outside [1, %d]", k, SPR_K_LIMIT);
        if (r->npix_cap * (int64_t)k > 0x7FFFFFFFll)
            return set_error(SPR_ERR_INVALID_ARG, "width*height*k exceeds 2^31 entries");
        r->k_fixed = k;
    } else if (mode == SPR_SPEC_ADAPTIVE) {
        if (k_max < 1 || k_max > SPR_K_LIMIT)
            return set_error(SPR_ERR_INVALID_ARG, "k_max = %d outside [1, %d]", k_max, SPR_K_LIMIT);
        r->k_max = k_max;
    } else if (per_ray_mode(mode)) {
        if (k_max < 1 || k_max > SPR_K_PER_RAY_LIMIT)
            return set_error(SPR_ERR_INVALID_ARG, "per-ray k_max = %d outside [1, %d]", k_max, SPR_K_PER_RAY_LIMIT);
        if (r->npix_cap * (int64_t)k_max > 0x7FFFFFFFll)
            return set_error(SPR_ERR_INVALID_ARG, "width*height*k_max exceeds 2^31 entries");
        if (mode == SPR_SPEC_LEARNED && !r->policy_set)
            return set_error(SPR_ERR_INVALID_ARG, "learned speculation needs a policy (spr_set_policy)");
        r->k_max = k_max;
    } else {
        return set_error(SPR_ERR_INVALID_ARG, "unknown speculation mode %d", mode);
    }
    // the captured pass graph holds the speculation layout and policy kernels
    if (per_ray_mode(mode) != per_ray_mode(r->spec_mode) || (mode != r->spec_mode && per_ray_mode(mode)))
        drop_graph(r);
    r->spec_mode = mode;
    r->need_raygen = true;
    r->params_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_warp_walk_threshold(spr_renderer *r, int64_t n_rays)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    if (n_rays < 0) return set_error(SPR_ERR_INVALID_ARG, "n_rays must be non-negative");
    const bool before = coop_walks_possible(r);
    r->coop_below = (uint32_t)std::min<int64_t>(n_rays, 0xFFFFFFFFll);
    if (coop_walks_possible(r) != before) drop_graph(r);   // the pass graph gains or loses the warp walks
    r->params_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_segment_walk(spr_renderer *r, int64_t lanes)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    if (lanes < 0) return set_error(SPR_ERR_INVALID_ARG, "negative lane budget");
    const uint32_t v = (uint32_t)std::min<int64_t>(lanes, 0x7FFFFFFFll);
    const bool before = coop_walks_possible(r);
    const bool had_seg = r->seg_threads != 0;
    r->seg_threads = v;
    // the pass graph gains or loses the segmented or the warp walks
    if ((v != 0) != had_seg || coop_walks_possible(r) != before) drop_graph(r);
    r->params_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_intersect_staging(spr_renderer *r, int on)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    if ((on != 0) != r->isect_staged) drop_graph(r);   // the pass graph holds the kernel
    r->isect_staged = on != 0;
    return SPR_OK;
}

extern "C" int spr_reset_cache(spr_renderer *r)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    r->cache_dirty = true;
    return SPR_OK;
}

extern "C" int spr_set_profiling(spr_renderer *r, int on)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    r->profiling = on != 0;
    return SPR_OK;
}

namespace {

// The whole render on the device, enqueued without waiting: the start graph
// (parameters, cache reset, ray generation, pass limit), then one launch of
// the pass graph whose while node runs passes until none is live.  Only
// first-time clears and the brick masks of a new isovalue are launched
// outside the graphs.  ev[0] marks the end of the render on `s`.
int submit_render(spr_renderer *r, cudaStream_t s, int max_passes)
{
    SPR_TRY(check_ready(r));
    if (max_passes < 1) return set_error(SPR_ERR_INVALID_ARG, "max_passes must be positive");
    if (r->profiling) return set_error(SPR_ERR_INVALID_ARG, "profiled renders are host-driven: turn profiling off");
    const bool fresh = r->need_raygen;
    SPR_TRY(ensure_entry_buffers(r, s));
    SPR_TRY(ensure_scan_scratch(r, s));
    struct Scope {
        Scope(int64_t *p) { g_launch_counter = p; }
        ~Scope() { g_launch_counter = nullptr; }
    } scope(&r->launches);
    if (fresh) r->launches = 0;
    if (r->cache_dirty && !r->cache_init) SPR_TRY(reset_cache(r, s));
    const uint32_t reset = r->cache_dirty ? 1u : 0u;
    if (fresh) SPR_TRY(update_occupancy(r, s));
    SPR_TRY(clear_bits_if_dirty(r, s));
    SPR_TRY(build_start_graph(r, fresh));
    SPR_TRY(build_graph(r));
    SPR_TRY(write_params(r, (uint32_t)max_passes, reset));
    if (fresh) {
        // no kernel of this renderer is in flight (the last render was
        // collected): start the mirror's pass count at zero, so that a query
        // before ray generation has run sees no pass of this render
        *(volatile uint32_t *)&r->h_ps->pass = 0u;
    }
    r->sub_before = *r->h_ps;
    SPR_CUDA_TRY(cudaEventRecord(r->ev[7], s));
    SPR_CUDA_TRY(cudaGraphLaunch(fresh ? r->gstart : r->glimit, s));
    SPR_CUDA_TRY(cudaEventRecord(r->ev_upload, s));
    SPR_CUDA_TRY(cudaEventRecord(r->ev[1], s));
    r->launches += fresh ? 4 : 2;
    r->cache_dirty = false;
    r->params_dirty = false;
    if (fresh) {
        r->need_raygen = false;
        r->pass = 0;
    }
    r->sub_fresh = fresh;
    r->sub_first = r->pass;
    SPR_CUDA_TRY(cudaGraphLaunch(r->gexec, s));
    SPR_CUDA_TRY(cudaEventRecord(r->ev[0], s));
    r->sub_stream = s;
    r->busy = true;
    return SPR_OK;
}

// Wait for a submitted render and fill its statistics.
int collect_render(spr_renderer *r, spr_render_stats *out, spr_pass_stats *per_pass)
{
    if (!r->busy) return set_error(SPR_ERR_INVALID_ARG, "no render was submitted");
    r->busy = false;
    const int first = r->sub_first;
    const bool fresh = r->sub_fresh;
    const PassState &before = r->sub_before;
    SPR_TRY(read_state(r, r->sub_stream));
    spr_render_stats rs;
    memset(&rs, 0, sizeof rs);
    const int passes = r->pass - first;
    const PassState &after = *r->h_ps;
    const bool same = !fresh;   // totals restart at ray generation
    rs.blocks_decoded = (int64_t)(after.tot_decoded - (same ? before.tot_decoded : 0));
    rs.entries = (int64_t)(after.tot_entries - (same ? before.tot_entries : 0));
    rs.evictions = (int64_t)(after.tot_evicted - (same ? before.tot_evicted : 0));
    rs.n_hits = (int64_t)(after.tot_hits - (same ? before.tot_hits : 0));
    int64_t attempts = (int64_t)after.attempts - (same ? (int64_t)before.attempts : 0);
    int nrec = std::max(0, std::min(first + passes, spr_renderer::kRecCap) - first);
    if (per_pass && nrec > 0) memcpy(per_pass, r->h_recs + first, sizeof(spr_pass_stats) * nrec);
    r->launches += (int64_t)r->graph_kernels * std::max<int64_t>(attempts, 1);
    float t_all = 0.f, t_ray = 0.f;
    cudaEventElapsedTime(&t_all, r->ev[7], r->ev[0]);
    cudaEventElapsedTime(&t_ray, r->ev[7], r->ev[1]);
    rs.ms_raygen = fresh ? t_ray : 0.f;
    rs.ms_total = t_all;
    rs.passes = passes;
    rs.n_rays = r->n_enter;
    rs.converged = r->n_live == 0;
    rs.bytes_decoded = rs.blocks_decoded * 256;
    rs.kernel_launches = r->launches;
    if (out) *out = rs;
    if (!rs.converged) return set_error(SPR_ERR_NOT_CONVERGED, "%d passes left rays live", passes);
    return SPR_OK;
}

}  // namespace

extern "C" int spr_render_pass(spr_renderer *r, spr_stream stream, spr_pass_stats *out)
{
    clear_error();
    if (r) SPR_TRY(check_idle(r));
    return do_pass(r, as_stream(stream), out);
}

extern "C" int spr_render_to_convergence(spr_renderer *r, spr_stream stream, int max_passes,
                                         spr_render_stats *out, spr_pass_stats *per_pass)
{
    clear_error();
    SPR_TRY(check_ready(r));
    SPR_TRY(check_idle(r));
    if (max_passes < 1) return set_error(SPR_ERR_INVALID_ARG, "max_passes must be positive");
    cudaStream_t s = as_stream(stream);
    spr_render_stats rs;
    memset(&rs, 0, sizeof rs);
    const bool fresh = r->need_raygen;
    int passes = 0;
    float ms = 0.f;
    if (r->profiling) {
        // host-driven passes with per-stage CUDA events
        while (passes < max_passes) {
            spr_pass_stats st;
            SPR_TRY(do_pass(r, s, &st));
            if (st.n_active == 0) break;
            if (per_pass && st.pass <= spr_renderer::kRecCap) per_pass[passes] = st;
            ++passes;
            rs.blocks_decoded += st.n_decoded;
            rs.entries += st.n_entries;
            rs.evictions += st.n_evicted;
            rs.n_hits += st.n_term_hit;
            ms += st.ms;
            if (r->n_live == 0) break;
        }
        rs.ms_raygen = fresh ? r->ms_raygen : 0.f;
        rs.ms_total = ms + rs.ms_raygen;
    } else {
        SPR_TRY(submit_render(r, s, max_passes));
        return collect_render(r, out, per_pass);
    }
    rs.passes = passes;
    rs.n_rays = r->n_enter;
    rs.converged = r->n_live == 0;
    rs.bytes_decoded = rs.blocks_decoded * 256;
    rs.kernel_launches = r->launches;
    if (out) *out = rs;
    if (!rs.converged) return set_error(SPR_ERR_NOT_CONVERGED, "%d passes left rays live", passes);
    return SPR_OK;
}

extern "C" int spr_render_submit(spr_renderer *r, spr_stream stream, int max_passes)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    return submit_render(r, as_stream(stream), max_passes);
}

extern "C" int spr_render_query(spr_renderer *r, int32_t *passes_done, int32_t *done)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    if (!r->busy) {
        if (passes_done) *passes_done = 0;
        if (done) *done = 1;
        return SPR_OK;
    }
    // the pass count is the mirror that end_pass_kernel writes to mapped
    // host memory after every pass; read after the event, so that a finished
    // render reports its final count
    cudaError_t e = cudaEventQuery(r->ev[0]);
    const uint32_t p = *(volatile const uint32_t *)&r->h_ps->pass;
    if (e != cudaSuccess && e != cudaErrorNotReady)
        return set_error(SPR_ERR_CUDA, "render query: %s", cudaGetErrorString(e));
    if (passes_done) *passes_done = (int32_t)std::max<int64_t>(0, (int64_t)p - r->sub_first);
    if (done) *done = e == cudaSuccess ? 1 : 0;
    return SPR_OK;
}

extern "C" int spr_render_collect(spr_renderer *r, spr_render_stats *out, spr_pass_stats *per_pass)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    return collect_render(r, out, per_pass);
}

extern "C" int spr_renderer_memory(const spr_renderer *r, size_t *device_bytes)
{
    clear_error();
    if (!r || !device_bytes) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    const DevBuf *bufs[] = {&r->state_in, &r->state_out, &r->status, &r->live[0], &r->live[1], &r->keys,
                            &r->fb_depth, &r->fb_rgba, &r->fb_block, &r->fb_cell, &r->fb_final, &r->rbid,
                            &r->erank, &r->E, &r->vis_bits, &r->act_bits, &r->vis_wpre, &r->bits_tsum,
                            &r->ivis, &r->iact, &r->nbrays, &r->obrays, &r->cache, &r->blk_slot,
                            &r->slot_blk, &r->lru[0], &r->lru[1], &r->touched, &r->miss, &r->victim,
                            &r->scan_status[0], &r->scan_status[1], &r->scan_status[2], &r->scan_ticket[0],
                            &r->scan_ticket[1], &r->scan_ticket[2], &r->ctr, &r->occ_fine, &r->occ_super,
                            &r->occ_box, &r->ps, &r->camd, &r->lbits, &r->kray, &r->koff, &r->eray, &r->policy,
                            &r->tr_count, &r->tr_taken, &r->tr_need};
    size_t n = 0;
    for (const DevBuf *b : bufs) n += b->bytes;
    *device_bytes = n;
    return SPR_OK;
}

extern "C" int spr_renderer_memory_estimate(const spr_volume *vol, int width, int height, int n_views,
                                            size_t cache_bytes, int spec_mode, int k, size_t *device_bytes)
{
    clear_error();
    if (!vol || !device_bytes || width < 1 || height < 1 || n_views < 1 || n_views > kMaxViews || k < 1)
        return set_error(SPR_ERR_INVALID_ARG, "bad estimate arguments");
    const VolGeom &g = vol->g;
    const int64_t np = (int64_t)width * height * n_views;
    const int64_t nwords = (g.nblocks + 31) / 32;
    const int64_t slots = (int64_t)(cache_bytes / 256);
    const int64_t cap = std::max<int64_t>(1, np * (spec_mode == SPR_SPEC_FIXED || per_ray_mode(spec_mode) ? k : 1));
    const int64_t act = std::min<int64_t>(g.nblocks, 8 * cap);
    int64_t ns = 1;
    for (int a = 0; a < 3; ++a) ns *= (g.nc[a] + 3) / 4;
    const int64_t scan_items = std::max({tiled_ray_count(width, height) * n_views, slots, nwords, cap, act,
                                         (int64_t)1});
    int64_t n = 12 * nwords + 8 * bits_tiles(nwords) + 4 * g.nblocks   // block bitmaps, block -> slot
                + 57 * np + 4 * (tiled_ray_count(width, height) * n_views / 32 + 1)   // per ray, bitmap
                + (8 * (g.ncoarse + ns) + 32) * n_views            // brick masks, occupied box
                + 269 * slots                                       // cache slots and their tables
                + 24 * cap + 8 + 12 * act                           // entries, requests
                + (per_ray_mode(spec_mode) ? 4 * cap + 8 * np : 0)  // per-ray counts, offsets, entry rays
                + 3 * 8 * (scan_tiles(scan_items) + 1) + 3 * 64     // look-back scratch
                + (int64_t)(sizeof(uint32_t) * C_COUNT + sizeof(PassState) + sizeof(DevParams) + 16);
    *device_bytes = (size_t)n;
    return SPR_OK;
}

extern "C" int spr_set_policy(spr_renderer *r, const float *params, float margin, int flags)
{
    clear_error();
    if (!r || !params) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    SPR_TRY(check_idle(r));
    if (!std::isfinite(margin)) return set_error(SPR_ERR_INVALID_ARG, "margin must be finite");
    for (int i = 0; i < mlp::kParams; ++i)
        if (!std::isfinite(params[i])) return set_error(SPR_ERR_INVALID_ARG, "policy parameter %d is not finite", i);
    if (flags & ~(SPR_POLICY_FLOOR | SPR_POLICY_FLOOR_AFTER_FIRST))
        return set_error(SPR_ERR_INVALID_ARG, "unknown policy flags 0x%x", flags);
    if (!r->policy.p) SPR_TRY(buf_alloc(r->policy, sizeof(float) * (mlp::kParams + 2), nullptr));
    // ordered after every earlier render of this renderer (they may read it)
    SPR_CUDA_TRY(cudaDeviceSynchronize());
    SPR_CUDA_TRY(cudaMemcpy(r->policy.p, params, sizeof(float) * mlp::kParams, cudaMemcpyHostToDevice));
    const float extra[2] = {margin, (flags & SPR_POLICY_FLOOR) ? 0.f : ((flags & SPR_POLICY_FLOOR_AFTER_FIRST) ? 1.f : -1.f)};
    SPR_CUDA_TRY(cudaMemcpy(r->policy.as<float>() + mlp::kParams, extra, sizeof extra, cudaMemcpyHostToDevice));
    r->policy_set = true;
    r->need_raygen = true;
    return SPR_OK;
}

extern "C" int spr_set_trace(spr_renderer *r, float *features, uint32_t *rays, uint32_t *consumed, int64_t capacity,
                             uint32_t sample_mod)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    SPR_TRY(check_idle(r));
    const bool on = features != nullptr;
    if (on && (!rays || !consumed || capacity < 1 || capacity > 0x7FFFFFFFll || sample_mod < 1))
        return set_error(SPR_ERR_INVALID_ARG, "bad trace buffers");
    if (on) {
        SPR_TRY(buf_reserve(r->tr_taken, sizeof(uint32_t) * r->npix_cap, nullptr));
        SPR_TRY(buf_reserve(r->tr_need, sizeof(uint32_t) * r->npix_cap, nullptr));
        if (!r->tr_count.p) SPR_TRY(buf_alloc(r->tr_count, sizeof(uint32_t), nullptr));
        SPR_CUDA_TRY(cudaMemset(r->tr_count.p, 0, sizeof(uint32_t)));
    }
    r->tr_feat = features;
    r->tr_ray = rays;
    r->tr_cons = consumed;
    r->tr_cap = (uint32_t)capacity;
    r->tr_mod = sample_mod;
    r->tr_from = 0;
    if (on != r->tracing || on) drop_graph(r);   // the pass graph holds the trace kernel and buffers
    r->tracing = on;
    r->need_raygen = true;
    return SPR_OK;
}

extern "C" int spr_trace_labels(spr_renderer *r, uint32_t *labels, int64_t *n_samples, spr_stream stream)
{
    clear_error();
    if (!r || !labels || !n_samples) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    SPR_TRY(check_idle(r));
    if (!r->tracing) return set_error(SPR_ERR_INVALID_ARG, "tracing is off");
    if (r->n_live != 0 || r->need_raygen)
        return set_error(SPR_ERR_INVALID_ARG, "labels need a converged render");
    cudaStream_t s = as_stream(stream);
    Trace T = make_trace(r);
    trace_label_kernel<<<grid_for(r->tr_cap, 256, 8), 256, 0, s>>>(T, r->tr_from, labels);
    SPR_CUDA_TRY(cudaGetLastError());
    uint32_t count = 0;
    SPR_CUDA_TRY(cudaMemcpyAsync(&count, r->tr_count.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SPR_CUDA_TRY(cudaStreamSynchronize(s));
    count = std::min(count, r->tr_cap);
    r->tr_from = count;
    *n_samples = count;
    return SPR_OK;
}

extern "C" int spr_get_framebuffer(spr_renderer *r, spr_framebuffer *out)
{
    clear_error();
    if (!r || !out) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    out->width = r->W;
    out->height = r->H * r->n_views;   // the views stacked top to bottom
    out->depth = r->fb_depth.as<float>();
    out->rgba = r->fb_rgba.as<uint32_t>();
    out->block = r->fb_block.as<uint32_t>();
    out->cell = r->fb_cell.as<uint64_t>();
    out->final_pass = r->fb_final.as<int32_t>();
    out->status = r->status.as<uint8_t>();
    return SPR_OK;
}

extern "C" int spr_read_framebuffer(spr_renderer *r, spr_stream stream, float *depth, uint32_t *rgba,
                                    uint32_t *block, uint64_t *cell, int32_t *final_pass, uint8_t *status)
{
    clear_error();
    if (!r) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer");
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)r->npix;
    if (depth) SPR_CUDA_TRY(cudaMemcpyAsync(depth, r->fb_depth.p, 4 * n, cudaMemcpyDeviceToHost, s));
    if (rgba) SPR_CUDA_TRY(cudaMemcpyAsync(rgba, r->fb_rgba.p, 4 * n, cudaMemcpyDeviceToHost, s));
    if (block) SPR_CUDA_TRY(cudaMemcpyAsync(block, r->fb_block.p, 4 * n, cudaMemcpyDeviceToHost, s));
    if (cell) SPR_CUDA_TRY(cudaMemcpyAsync(cell, r->fb_cell.p, 8 * n, cudaMemcpyDeviceToHost, s));
    if (final_pass) SPR_CUDA_TRY(cudaMemcpyAsync(final_pass, r->fb_final.p, 4 * n, cudaMemcpyDeviceToHost, s));
    if (status) SPR_CUDA_TRY(cudaMemcpyAsync(status, r->status.p, n, cudaMemcpyDeviceToHost, s));
    SPR_CUDA_TRY(cudaStreamSynchronize(s));
    return SPR_OK;
}

// ------------------------------------------------------------------- scan
namespace {
int scan_impl(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, int64_t withhold, int64_t spin,
              cudaStream_t s)
{
    if (n < 0 || (n > 0 && (!in || !out))) return set_error(SPR_ERR_INVALID_ARG, "bad scan arguments");
    if (n > 0xFFFFFFFFll) return set_error(SPR_ERR_INVALID_ARG, "scan longer than 2^32");
    DevBuf status, ticket, flags;
    int rc = SPR_OK;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        buf_free(status, s);
        buf_free(ticket, s);
        buf_free(flags, s);
    };
    if ((rc = buf_alloc(status, sizeof(unsigned long long) * (scan_tiles(n) + 1), s)) ||
        (rc = buf_alloc(ticket, 64, s)) || (rc = buf_alloc(flags, 64, s))) {
        cleanup();
        return rc;
    }
    if (cudaMemsetAsync(flags.p, 0, 64, s) != cudaSuccess || cudaMemsetAsync(ticket.p, 0, 64, s) != cudaSuccess ||
        cudaMemsetAsync(status.p, 0, status.bytes, s) != cudaSuccess) {
        cleanup();
        return set_error(SPR_ERR_CUDA, "memset failed");
    }
    rc = run_compact(status, ticket, flags.as<uint32_t>(), n, nullptr, ArrayCount{in, nullptr}, ArrayEmit{out},
                     total, s, spin, withhold);
    uint32_t f = 0;
    if (rc == SPR_OK) {
        cudaError_t e = cudaMemcpyAsync(&f, flags.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "scan: %s", cudaGetErrorString(e));
    }
    cleanup();
    if (rc == SPR_OK && f) rc = set_error(SPR_ERR_DEVICE_TIMEOUT, "a look-back wait gave up after its poll limit");
    return rc;
}
}  // namespace

extern "C" int spr_exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                                      spr_stream stream)
{
    clear_error();
    return scan_impl(in, out, n, total, -1, kDefaultSpinLimit, as_stream(stream));
}

extern "C" int spr_debug_scan_withhold(const uint32_t *in, uint32_t *out, int64_t n, int64_t withhold_tile,
                                       int64_t spin_limit, spr_stream stream)
{
    clear_error();
    if (spin_limit < 1) return set_error(SPR_ERR_INVALID_ARG, "spin_limit must be positive");
    return scan_impl(in, out, n, nullptr, withhold_tile, spin_limit, as_stream(stream));
}

// ------------------------------------------------------------------ batch
// Several renderers -- of different volumes, image sizes and view counts --
// rendered by one graph launch.  Each keeps everything its own render uses
// (cache, brick masks, wavefront, scan scratch, pass state); the graph holds,
// per renderer, the start of its render (parameter copy, ray generation) as
// a child graph followed by its pass loop (a conditional while node over one
// pass attempt).  The branches have no edges between them, so the device runs
// the renders concurrently, and the small passes of one overlap the others'.
struct spr_batch {
    std::vector<spr_renderer *> rs;
    std::vector<uint64_t> gens;        // each renderer's graph generation at capture
    std::vector<int64_t> n_slots;      // and its cache size
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_drop(spr_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

int batch_build(spr_batch *b)
{
    batch_drop(b);
    cudaGraph_t g = nullptr;
    SPR_CUDA_TRY(cudaGraphCreate(&g, 0));
    int rc = SPR_OK;
    for (spr_renderer *r : b->rs) {
        cudaGraph_t sg = nullptr;
        if ((rc = capture_start_graph(r, true, &sg)) != SPR_OK) break;
        cudaGraphNode_t start = nullptr;
        cudaError_t e = cudaGraphAddChildGraphNode(&start, g, nullptr, 0, sg);
        cudaGraphDestroy(sg);   // the node holds its own copy
        cudaGraphConditionalHandle h;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&loop, g, &start, nullptr, 1, &cp);
        if (e != cudaSuccess) {
            rc = set_error(SPR_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
            break;
        }
        e = cudaStreamBeginCaptureToGraph(r->cap_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        const int64_t saved = r->launches;
        int rc2 = e == cudaSuccess ? enqueue_attempt(r, r->cap_stream, false, h, 1) : SPR_OK;
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(r->cap_stream, &captured) : e;
        r->launches = saved;
        if (rc2 != SPR_OK) {
            rc = rc2;
            break;
        }
        if (e != cudaSuccess || e2 != cudaSuccess) {
            rc = set_error(SPR_ERR_CUDA, "batch pass capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
            break;
        }
    }
    if (rc == SPR_OK) {
        cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            rc = set_error(SPR_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    if (rc != SPR_OK) {
        cudaGraphDestroy(g);
        return rc;
    }
    b->graph = g;
    for (size_t i = 0; i < b->rs.size(); ++i) {
        b->gens[i] = b->rs[i]->graph_gen;
        b->n_slots[i] = b->rs[i]->n_slots;
    }
    return SPR_OK;
}

}  // namespace

extern "C" int spr_batch_create(spr_renderer *const *renderers, int n, spr_batch **out)
{
    clear_error();
    if (!out || !renderers || n < 1) return set_error(SPR_ERR_INVALID_ARG, "a batch needs renderers");
    if (n > 256) return set_error(SPR_ERR_INVALID_ARG, "at most 256 renderers in a batch");
    for (int i = 0; i < n; ++i) {
        if (!renderers[i]) return set_error(SPR_ERR_INVALID_ARG, "NULL renderer %d", i);
        for (int j = 0; j < i; ++j)
            if (renderers[j] == renderers[i]) return set_error(SPR_ERR_INVALID_ARG, "renderer %d is listed twice", i);
    }
    spr_batch *b = new (std::nothrow) spr_batch;
    if (!b) return set_error(SPR_ERR_OUT_OF_MEMORY, "host allocation failed");
    b->rs.assign(renderers, renderers + n);
    b->gens.assign((size_t)n, ~0ull);
    b->n_slots.assign((size_t)n, -1);
    *out = b;
    return SPR_OK;
}

extern "C" int spr_batch_destroy(spr_batch *b)
{
    clear_error();
    if (!b) return SPR_OK;
    cudaDeviceSynchronize();
    batch_drop(b);
    delete b;
    return SPR_OK;
}

extern "C" int spr_batch_render(spr_batch *b, spr_stream stream, int max_passes, spr_render_stats *stats)
{
    clear_error();
    if (!b) return set_error(SPR_ERR_INVALID_ARG, "NULL batch");
    if (max_passes < 1) return set_error(SPR_ERR_INVALID_ARG, "max_passes must be positive");
    cudaStream_t s = as_stream(stream);
    for (spr_renderer *r : b->rs) {
        SPR_TRY(check_ready(r));
        SPR_TRY(check_idle(r));
        if (r->profiling) return set_error(SPR_ERR_INVALID_ARG, "profiled renders are host-driven: turn profiling off");
        if (!r->need_raygen)
            return set_error(SPR_ERR_INVALID_ARG, "a batch render starts every render at ray generation: "
                                                  "set a camera or an isovalue of each renderer first");
    }
    for (spr_renderer *r : b->rs) {
        SPR_TRY(ensure_entry_buffers(r, s));
        SPR_TRY(ensure_scan_scratch(r, s));
    }
    bool stale = !b->exec;
    for (size_t i = 0; i < b->rs.size(); ++i)
        stale |= b->gens[i] != b->rs[i]->graph_gen || b->n_slots[i] != b->rs[i]->n_slots;
    if (stale) SPR_TRY(batch_build(b));
    for (spr_renderer *r : b->rs) {
        r->launches = 0;
        if (r->cache_dirty && !r->cache_init) SPR_TRY(reset_cache(r, s));
        const uint32_t reset = r->cache_dirty ? 1u : 0u;
        SPR_TRY(update_occupancy(r, s));
        SPR_TRY(clear_bits_if_dirty(r, s));
        SPR_TRY(write_params(r, (uint32_t)max_passes, reset));
        *(volatile uint32_t *)&r->h_ps->pass = 0u;
        r->sub_before = *r->h_ps;
        SPR_CUDA_TRY(cudaEventRecord(r->ev[7], s));
        SPR_CUDA_TRY(cudaEventRecord(r->ev[1], s));   // no separate ray-generation time in a batch
    }
    SPR_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    for (spr_renderer *r : b->rs) {
        SPR_CUDA_TRY(cudaEventRecord(r->ev_upload, s));
        SPR_CUDA_TRY(cudaEventRecord(r->ev[0], s));
        r->launches += 4;   // the start graph's kernels
        r->cache_dirty = false;
        r->params_dirty = false;
        r->need_raygen = false;
        r->pass = 0;
        r->sub_fresh = true;
        r->sub_first = 0;
        r->sub_stream = s;
        r->busy = true;
    }
    int rc = SPR_OK;
    for (size_t i = 0; i < b->rs.size(); ++i) {
        struct Scope {
            Scope(int64_t *p) { g_launch_counter = p; }
            ~Scope() { g_launch_counter = nullptr; }
        } scope(&b->rs[i]->launches);
        int ri = collect_render(b->rs[i], stats ? &stats[i] : nullptr, nullptr);
        if (rc == SPR_OK) rc = ri;
    }
    return rc;
}
