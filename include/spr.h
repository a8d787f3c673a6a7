/*
 * spr.h -- C ABI of the GB300 speculative progressive isosurface raycaster.
 *
 * The method is the one of Usher, Dyken and Kumar, "Speculative Progressive
 * Raycasting for Memory Constrained Isosurface Visualization of Massive
 * Volumes" (arXiv 2309.10212): a wavefront of rays is advanced through a
 * block-compressed volume one pass at a time; each pass (Fig. 2, Sec. 3, 4)
 *   (a) advances every live ray through the two-level macrocell grid to its
 *       next k blocks whose value range holds the isovalue (Sec. 3.3, 4.1),
 *   (b) marks those blocks visible and their +x/+y/+z neighbours active
 *       (Sec. 3.4), groups the ray-block entries by block (Sec. 3.6, 4.2),
 *   (c) decompresses the active blocks that are not cached into a fixed
 *       budget LRU cache (Sec. 3.5),
 *   (d) intersects each entry's ray with the trilinear isosurface inside its
 *       block (Sec. 3.7, 4.3) and keeps each ray's earliest hit (Sec. 4.4),
 *   (e) compacts the rays still live for the next pass (Sec. 3, step f).
 * k is a fixed speculation count or floor(w*h / N_Act) capped at k_max
 * (Sec. 4).  Every step runs in CUDA kernels on one GPU; the host reads one
 * small counter record per pass.
 *
 * Conventions
 *   - Every function returns an int status: SPR_OK (0) or a negative
 *     SPR_ERR_* code.  Nothing throws or exits across the ABI.  The text of
 *     the most recent error of the calling thread is spr_last_error().
 *   - Handles are opaque; one host thread uses a handle at a time.
 *   - spr_stream is a cudaStream_t passed as void* (NULL: the legacy default
 *     stream).  Work is ordered on that stream; functions that return
 *     statistics synchronise it.
 *   - "device" pointers are CUDA device memory of the current device; "host"
 *     pointers are ordinary (or pinned) host memory.  Caller buffers are only
 *     borrowed for the duration of the call unless stated otherwise.
 *   - Device memory the library needs is taken from the allocator set with
 *     spr_set_allocator (default: cudaMalloc/cudaFree); allocation failure is
 *     SPR_ERR_OUT_OF_MEMORY.
 *
 * Geometry (Sec. 3.2, 3.7): voxel (x,y,z) sits at point (x,y,z); the domain is
 * [0,Dx-1]x[0,Dy-1]x[0,Dz-1]; cell (x,y,z) is the unit cube with that lower
 * corner and the field inside is the trilinear interpolant of its corners.
 * The ray of pixel (i,j) (j = 0 the bottom row, pixel id i + W*j) is
 * eye + t*d with d = (p00 + (i+0.5f)*du) + (j+0.5f)*dv evaluated per
 * component in IEEE single precision without fused multiply-add; the hit is
 * the first point along the ray where the interpolant equals the isovalue.
 */
#ifndef SPR_H
#define SPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define SPR_OK                    0
#define SPR_ERR_INVALID_ARG      -1  /* a bad pointer, size, camera or mode          */
#define SPR_ERR_OUT_OF_MEMORY    -2  /* the allocator returned NULL                  */
#define SPR_ERR_CACHE_TOO_SMALL  -3  /* cache budget below 8 slots (8 x 256 bytes)   */
#define SPR_ERR_CUDA             -4  /* a CUDA runtime call failed                   */
#define SPR_ERR_DEVICE_TIMEOUT   -5  /* a bounded device-side wait gave up           */
#define SPR_ERR_NOT_CONVERGED    -6  /* max_passes reached with rays still live      */
#define SPR_ERR_NOT_IMPLEMENTED  -7
#define SPR_ERR_NO_DEVICE        -8  /* no CUDA device / wrong architecture          */
#define SPR_ERR_DEVICE_ERROR     -9  /* a kernel reported an internal error flag     */

typedef void *spr_stream;
typedef struct spr_volume spr_volume;
typedef struct spr_renderer spr_renderer;

/* text of the calling thread's most recent error ("" if none) */
const char *spr_last_error(void);
/* fixed description of a status code */
const char *spr_status_string(int status);
/* library version, e.g. 10000 for 1.0.0 */
int spr_version(void);

/* ------------------------------------------------------------- allocator */
/* Process-wide device allocator for all library-owned memory.  alloc returns
 * a device pointer of at least `bytes` (256-byte aligned) or NULL; free
 * releases it.  `stream` is the stream the memory is first used on.  Passing
 * NULL for both restores cudaMalloc/cudaFree.  Set it while no handle is
 * alive; memory is freed with the allocator that allocated it. */
typedef void *(*spr_alloc_fn)(size_t bytes, spr_stream stream, void *ctx);
typedef void (*spr_free_fn)(void *ptr, size_t bytes, spr_stream stream, void *ctx);
int spr_set_allocator(spr_alloc_fn alloc, spr_free_fn free_fn, void *ctx);

/* ------------------------------------------------------------------ codec */
/*
 * FRC4: the fixed-rate 4^3 block codec that stands in for the ZFP
 * fixed-rate mode the paper decompresses on the GPU (Sec. 3.1, 3.5).  At rate
 * R (1..32 bits per value) every block is 8*R bytes, block b (x-fastest over
 * the nb = ceil(D/4) block grid) at byte 8*R*b.  A block is: a 1 bit "block
 * is nonzero" (else all zero), 8 bits emax+127 (emax = largest frexp exponent,
 * clamped to >= -100), then bit planes 29..0 of the negabinary, sequency-
 * ordered coefficients of a two-level integer S-transform along x, y, z of
 * q = round-half-even(x * 2^(24-emax)), each plane as refinement bits of the
 * significant prefix followed by group tests, cut at the budget.  Bit k of a
 * block is bit k&7 of byte k>>3.  Partial blocks repeat the last voxel.
 */
#define SPR_CODEC_FRC4 1

/* Compress a device volume (x fastest, dims[0]*dims[1]*dims[2] values) into
 * out (device, nb[0]*nb[1]*nb[2]*8*rate bytes).  u8 voxels are read as
 * (float)u / 255.0f.  Non-finite input -> SPR_ERR_INVALID_ARG. */
int spr_encode_f32(const float *vol, const int32_t dims[3], int rate, uint8_t *out,
                   spr_stream stream);
int spr_encode_u8(const uint8_t *vol, const int32_t dims[3], int rate, uint8_t *out,
                  spr_stream stream);

/* Decompress n blocks of a device block stream into out (device, n*64
 * floats, block-major, value index x + 4y + 16z).  ids (device, n entries)
 * selects the blocks; ids == NULL means blocks 0..n-1.  The block id must be
 * below n_blocks (the stream's block count); larger ids are an error. */
int spr_decode_blocks(const uint8_t *blocks, int64_t n_blocks, int rate, const uint32_t *ids,
                      int64_t n, float *out, spr_stream stream);

/* Decompress n blocks of a volume into out (device, n*64 floats, as
 * spr_decode_blocks), the way the renderer decodes its cache misses (Sec.
 * 3.5): the entries are grouped by the number of bit planes their parse
 * reads (recorded by spr_create_volume) so that a warp's lanes parse alike.
 * The values are identical to spr_decode_blocks'.  ids (device, n entries)
 * selects the blocks, ids == NULL means blocks 0..n-1; an id beyond the
 * volume's block count is SPR_ERR_INVALID_ARG.  n == 0 does nothing (out
 * may then be NULL).  Synchronises `stream`. */
int spr_volume_decode_blocks(const spr_volume *vol, const uint32_t *ids, int64_t n, float *out,
                             spr_stream stream);

/* ----------------------------------------------------------------- volume */
typedef struct {
    int32_t dims[3];        /* voxels per axis, each in [2, 4096]              */
    int32_t rate;           /* bits per value, 1..32                           */
    int32_t codec;          /* SPR_CODEC_FRC4                                  */
} spr_volume_desc;

/* Create a volume from its compressed blocks (Sec. 3.1).  blocks points to
 * nbytes = nb[0]*nb[1]*nb[2]*8*rate bytes, in device memory if
 * blocks_on_device, else in host memory.  The library copies them, decodes
 * every block once to get its value range, and builds the fine (per block)
 * and coarse (per 4^3 blocks) macrocell grids, each range combined with the
 * +x/+y/+z neighbours' (Sec. 3.1).  The same pass records, one byte per
 * block, how many bit planes the block's parse reads; the renderer's decoder
 * groups its cache misses by that count (no counterpart in the paper; the
 * decoded values do not depend on it).  Ordered on `stream`; returns after the
 * work is enqueued.  *out is owned by the caller (spr_destroy_volume). */
int spr_create_volume(const spr_volume_desc *desc, const void *blocks, size_t nbytes,
                      int blocks_on_device, spr_stream stream, spr_volume **out);
int spr_destroy_volume(spr_volume *vol);

/* Copy the volume's range grids to host memory: fine = nb blocks x (min,max),
 * coarse = ceil(nb/4) cells x (min,max), float pairs (either may be NULL).
 * Synchronises `stream`. */
int spr_volume_ranges(const spr_volume *vol, float *fine_host, float *coarse_host,
                      spr_stream stream);
/* block-grid and coarse-grid sizes; either pointer may be NULL */
int spr_volume_shape(const spr_volume *vol, int64_t nb[3], int64_t nc[3]);

/* The decode-everything-active alternative the progressive method is
 * measured against (Sec. 5.3 compares with a renderer that decompresses
 * every block the isovalue can touch): *n_active = blocks whose fine range
 * holds iso; *n_needed = those and their +x/+y/+z face, edge and corner
 * neighbours, whose values enter the active blocks' cells (what such a
 * renderer must decode).  Either pointer may be NULL; synchronises
 * `stream`. */
int spr_count_active_blocks(const spr_volume *vol, float iso, int64_t *n_active, int64_t *n_needed,
                            spr_stream stream);

/* --------------------------------------------------------------- renderer */
#define SPR_SPEC_FIXED    0   /* k = the given count every pass                */
#define SPR_SPEC_ADAPTIVE 1   /* k = min(k_max, floor(w*h / N_Act)) (Sec. 4)   */
/* Per-ray speculation: every live ray takes its own count k_i in [1, k_max]
 * each pass (the paper's future work, Sec. 6: a per-ray speculation count).
 * The image does not depend on the counts; only the passes and the blocks
 * decoded do.  Every attempt of a pass caps k_i by kk, which starts at k_max
 * and halves when the pass overflows the cache, as k does in the rules above.
 *
 * SPR_SPEC_HASHED, a model-free per-ray count: in pass P (1-based), the ray
 * with id q (view * w*h + y*w + x) takes k_i = min(kk, 1 + (h mod k_max)),
 * where, in unsigned 32-bit arithmetic,
 *     h  = (q * 0x9E3779B1) ^ (P * 0x85EBCA77);
 *     h ^= h >> 15;  h *= 0x2C1B3C6D;  h ^= h >> 12; */
#define SPR_SPEC_HASHED   2   /* k_i from the hash of (ray, pass) above                  */
#define SPR_SPEC_LEARNED  3   /* k_i from the renderer's policy MLP (spr_set_policy)              */
#define SPR_K_LIMIT       4096
#define SPR_K_PER_RAY_LIMIT 64

typedef struct {
    int32_t pass;           /* 1-based pass index since the last reset          */
    int32_t k;              /* speculation count from the rule                  */
    int32_t k_used;         /* after halving on cache overflow                  */
    int32_t retries;        /* passes redone because the cache was too small    */
    int64_t n_active;       /* live rays at pass start (N_Act)                  */
    int64_t n_processed;    /* live rays taken this pass                        */
    int64_t n_entries;      /* non-empty ray-block entries (speculated included)*/
    int64_t n_visible;      /* unique visible blocks (I_BVis)                   */
    int64_t n_requested;    /* unique active blocks: visible + neighbours       */
    int64_t n_decoded;      /* cache misses = blocks decompressed               */
    int64_t n_evicted;      /* misses that replaced a cached block              */
    int64_t n_term_hit;     /* rays finished with a hit this pass               */
    int64_t n_term_miss;    /* rays that left the volume this pass              */
    int64_t n_active_after; /* live rays after the pass                         */
    double  utilization;    /* n_entries / (w*h) (Table 2)                      */
    float   ms;             /* device time of the pass (profiling on, else 0)   */
    float   ms_stage[6];    /* traverse, group, cache, decode, intersect, resolve*/
    int64_t n_steps;        /* block and skip steps of all walks in the pass    */
    int64_t max_steps;      /* steps of the longest walk in the pass            */
} spr_pass_stats;

typedef struct {
    int32_t passes;
    int32_t converged;      /* 1 when no live ray is left                       */
    int64_t blocks_decoded; /* over all passes                                  */
    int64_t bytes_decoded;  /* blocks_decoded * 256                             */
    int64_t entries;        /* ray-block tests over all passes                  */
    int64_t evictions;
    int64_t n_rays;         /* rays that entered the volume                     */
    int64_t n_hits;
    float   ms_total;       /* device time from ray generation to convergence   */
    float   ms_raygen;
    int64_t kernel_launches;/* kernels the library launched for this render     */
} spr_render_stats;

/* Framebuffer (device, owned by the renderer; valid until the next set_* or
 * render call).  Pixel p = i + W*j. */
typedef struct {
    int32_t   width, height;
    float    *depth;        /* t*|d| in voxels; +inf where no hit               */
    uint32_t *rgba;         /* grey shade g as g|g<<8|g<<16|255<<24; 0 = no hit  */
    uint32_t *block;        /* hit block id (x-fastest over nb) or 0xFFFFFFFF   */
    uint64_t *cell;         /* hit cell x + Dx*(y + Dy*z) or ~0                 */
    int32_t  *final_pass;   /* pass in which the pixel became final; 0 = never  */
    uint8_t  *status;       /* 0 live, 1 hit, 2 left the volume / missed it     */
} spr_framebuffer;

/* Create a renderer of a width x height image for vol (which must outlive
 * it).  Defaults: isovalue 0.5, adaptive speculation with k_max 64, cache
 * budget 256 MiB, no camera (render calls fail until spr_set_camera). */
int spr_create_renderer(spr_volume *vol, int width, int height, spr_renderer **out);
int spr_destroy_renderer(spr_renderer *r);

/* Camera (Sec. 3.2): float triples eye, p00, du, dv (see the geometry note
 * above).  Each eye component must be a multiple of 1/256 with magnitude
 * below 16384, and every component of p00, du, dv zero or of magnitude in
 * [2^-40, 2^40]; otherwise SPR_ERR_INVALID_ARG.  With these bounds every
 * plane offset X - eye is exact in single precision, which the exact
 * traversal predicates rely on.  Restarts the render. */
int spr_set_camera(spr_renderer *r, const float eye[3], const float p00[3], const float du[3],
                   const float dv[3]);
/* isovalue (finite) of every view; restarts the render (the cache contents
 * are kept) */
int spr_set_isovalue(spr_renderer *r, float iso);
/* Batched rendering (no counterpart in the paper, which renders one view):
 * n_views (1..64) views of the volume are rendered as one wavefront -- their
 * rays share the passes, the speculation budget (k = min(k_max,
 * floor(n_views*w*h / N_Act))) and the block cache, so a block decoded for
 * one view serves all.  Each view's image equals its single-view render.
 * The framebuffer holds the views stacked top to bottom (height * n_views
 * rows); ray / pixel ids are view * w * h + y * w + x.  The per-pixel
 * buffers and captured graphs grow to the largest count set so far (that
 * reallocation synchronises the device); a count within that capacity
 * reuses them (views past n_views generate no rays).  Restarts the render;
 * every view needs a camera (spr_set_camera sets view 0, spr_set_view
 * any). */
int spr_set_view_count(spr_renderer *r, int n_views);
/* camera (as spr_set_camera) and isovalue of view `view` < n_views */
int spr_set_view(spr_renderer *r, int view, const float eye[3], const float p00[3], const float du[3],
                 const float dv[3], float iso);
/* cache budget in bytes; slots = bytes / 256, at least 8, else
 * SPR_ERR_CACHE_TOO_SMALL.  Empties the cache and restarts the render. */
int spr_set_cache_budget(spr_renderer *r, size_t bytes);
/* mode SPR_SPEC_FIXED with 1 <= k <= SPR_K_LIMIT, SPR_SPEC_ADAPTIVE with
 * 1 <= k_max <= SPR_K_LIMIT (k ignored), or a per-ray mode with 1 <= k_max
 * <= SPR_K_PER_RAY_LIMIT (SPR_SPEC_LEARNED needs a policy set first).  In a
 * per-ray mode a pass that overflows the cache is redone with every count
 * capped at half the previous cap, then (at 1) with half the rays.
 * Restarts the render. */
int spr_set_speculation(spr_renderer *r, int mode, int k, int k_max);
/* Traversal tuning (no counterpart in the paper, results unchanged): passes
 * with fewer than n_rays live rays walk one ray per warp, larger passes one
 * ray per thread (default 16384; 0 = never one per warp).  Both walks visit
 * the same blocks in the same order (Sec. 3.3).  Takes effect at the next
 * render or pass. */
int spr_set_warp_walk_threshold(spr_renderer *r, int64_t n_rays);
/* Segmented walk (no counterpart in the paper, results unchanged): a pass of
 * n live rays with lanes / n >= 2 gives each ray a group of G lanes (G the
 * largest power of two <= min(lanes / n, 32)).  The ray's remaining path is
 * cut at block planes of the axis along which its direction is largest into
 * G parts of equal block count; each lane walks one part (the first resumes
 * the saved walk, the others start at the exact crossing time of their first
 * plane) and the group keeps the first k visible blocks in walk order -- the
 * same blocks, in the same order, as the one-lane walk (Sec. 3.3).  Passes
 * with lanes / n < 2 use the walks above.  Default 262144 lanes; 0 turns
 * it off.  Takes effect at the next render or pass. */
int spr_set_segment_walk(spr_renderer *r, int64_t lanes);
/* Intersection variant (results unchanged): on = stage each visible block's
 * 5^3 dual grid in shared memory and intersect its entries from there, as
 * Sec. 3.7's work groups do; off (the default) = read each cell's corners
 * from the cache slots.  Takes effect at the next render or pass. */
int spr_set_intersect_staging(spr_renderer *r, int on);
/* empty the block cache (the next pass decodes from scratch) */
int spr_reset_cache(spr_renderer *r);
/* per-pass CUDA-event timing of the stages (adds host synchronisation) */
int spr_set_profiling(spr_renderer *r, int on);

/* Run one pass (steps a-e above) on `stream`.  The first pass after a set_*
 * call also generates the rays.  On a converged render it does nothing and
 * reports n_active = 0.  Synchronises `stream` once (to read the pass's
 * counters).  out may be NULL. */
int spr_render_pass(spr_renderer *r, spr_stream stream, spr_pass_stats *out);

/* Run passes until no ray is live or max_passes passes ran (then
 * SPR_ERR_NOT_CONVERGED, with the partial image valid).  Without profiling
 * the whole render is one CUDA graph launch (a conditional while node over
 * passes) and the host waits once at the end.  per_pass (may be NULL)
 * receives one record per pass, for the first 4096 passes since ray
 * generation; the totals in out cover every pass.  out may be NULL. */
int spr_render_to_convergence(spr_renderer *r, spr_stream stream, int max_passes,
                              spr_render_stats *out, spr_pass_stats *per_pass);

/* device pointers of the current framebuffer */
int spr_get_framebuffer(spr_renderer *r, spr_framebuffer *out);

/* Copy the framebuffer to host buffers of width*height entries each (any may
 * be NULL); synchronises `stream`. */
int spr_read_framebuffer(spr_renderer *r, spr_stream stream, float *depth, uint32_t *rgba,
                         uint32_t *block, uint64_t *cell, int32_t *final_pass,
                         uint8_t *status);

/* ------------------------------------------------------ asynchronous render */
/* The render of spr_render_to_convergence (without profiling) enqueued on
 * `stream` without waiting: ray generation when the render restarts, then
 * passes until no ray is live or max_passes ran.  Until spr_render_collect,
 * the renderer accepts only spr_render_query, spr_render_collect,
 * spr_get_framebuffer and spr_destroy_renderer (other calls return
 * SPR_ERR_INVALID_ARG); the framebuffer is complete once `stream` reaches
 * the end of the render.  Renders of different renderers submitted on
 * different streams overlap on the device.  With profiling on:
 * SPR_ERR_INVALID_ARG. */
int spr_render_submit(spr_renderer *r, spr_stream stream, int max_passes);
/* Non-blocking progress of a submitted render: *passes_done = passes
 * completed so far (read from the pass-state mirror the device writes into
 * mapped host memory after every pass, the progressive display of Sec. 3),
 * *done = 1 when the device has finished the render (either may be NULL).
 * Without a submitted render: 0 passes, done. */
int spr_render_query(spr_renderer *r, int32_t *passes_done, int32_t *done);
/* Wait for the submitted render and report it as spr_render_to_convergence
 * does (same statuses, e.g. SPR_ERR_NOT_CONVERGED). */
int spr_render_collect(spr_renderer *r, spr_render_stats *out, spr_pass_stats *per_pass);
/* Batched renders of several volumes (no counterpart in the paper, which
 * renders one view of one volume; Sec. 4's shared speculation budget and
 * cache already generalise to the views of one renderer).  A batch lists n
 * renderers -- of the same or different volumes, image sizes, view counts
 * and cache budgets -- and spr_batch_render renders all of them with ONE
 * graph launch on `stream`: per renderer, the start of its render (ray
 * generation) as a child graph, then its pass loop as a conditional while
 * node; the branches are independent, so the renders run concurrently.
 * Each renderer keeps its own block cache, brick masks and wavefront, and
 * its images equal those of its own spr_render_to_convergence.  Every
 * renderer must have a camera and start a fresh render (a set_camera,
 * set_view or set_isovalue since its last render), else SPR_ERR_INVALID_ARG.
 * stats (n entries, may be NULL) receives each renderer's statistics; its
 * ms_total is the batch's device time.  Blocks until the batch is done.  The
 * graph is captured at the first render and again when a renderer's buffers
 * or cache size changed.  The renderers must outlive the batch and are not
 * used elsewhere while spr_batch_render runs; a renderer may be in several
 * batches. */
typedef struct spr_batch spr_batch;
int spr_batch_create(spr_renderer *const *renderers, int n, spr_batch **out);
int spr_batch_destroy(spr_batch *b);
int spr_batch_render(spr_batch *b, spr_stream stream, int max_passes, spr_render_stats *stats);

/* device bytes the renderer holds now (buffers grown by earlier renders
 * included) */
int spr_renderer_memory(const spr_renderer *r, size_t *device_bytes);
/* device bytes a renderer of this shape holds after its first render:
 * n_views views of width x height, cache_bytes of block cache, speculation
 * mode and fixed k (ignored when adaptive) */
int spr_renderer_memory_estimate(const spr_volume *vol, int width, int height, int n_views,
                                 size_t cache_bytes, int spec_mode, int k, size_t *device_bytes);

/* ----------------------------------------------------------------- serving */
/*
 * A render service (no counterpart in the paper, which renders one view at a
 * time): requests -- a volume, an image size, a camera and an isovalue --
 * are queued and admitted while an in-flight slot (one CUDA stream each, at
 * most max_inflight) is free and the device memory budget holds the renderer
 * the request needs.  Renderers (block cache, wavefront buffers and captured
 * pass graphs) are pooled and reused across requests, so a volume's cache
 * stays warm between requests; when the budget is short, idle renderers are
 * released, least recently used first (those no queued request wants go
 * first); a request whose shape has a busy renderer waits for it instead of
 * releasing others.  Queued requests of the same volume and image size are
 * merged, oldest first and up to max_batch and the renderer's view capacity,
 * into one batched render (spr_set_view_count): one wavefront, one
 * speculation budget, one cache.  Requests of one shape start in arrival
 * order; the oldest request that can start does, so a shape whose
 * renderers are busy does not hold up the others.  Every result equals the
 * request's single-view render (the
 * image does not depend on the cache state, the speculation count or the
 * batch).  The scheduler runs on the calling host thread inside
 * spr_server_poll; one thread uses a server at a time.  Creating a pooled
 * renderer allocates device memory and synchronises the device, so the
 * first request of each (volume, size, batch) shape waits for the renders
 * in flight.
 */
typedef struct spr_server spr_server;

typedef struct {
    size_t  memory_bytes;   /* budget for the pooled renderers' device memory */
    int32_t max_inflight;   /* renders on the device at once, 1..64           */
    int32_t max_batch;      /* requests merged into one render, 1..64         */
    int32_t spec_mode;      /* SPR_SPEC_FIXED or SPR_SPEC_ADAPTIVE            */
    int32_t k, k_max;       /* as spr_set_speculation                          */
    int32_t max_passes;     /* per render                                      */
} spr_server_desc;

typedef struct {
    int32_t volume;             /* id from spr_server_add_volume                */
    int32_t width, height;
    float   eye[3], p00[3], du[3], dv[3];   /* as spr_set_camera              */
    float   iso;
    double  t_arrival;          /* seconds on spr_server_clock; < 0: now        */
    /* caller-owned device buffers of width*height entries (any may be NULL),
     * filled by the device when the request completes (as spr_framebuffer) */
    float    *depth;
    uint32_t *rgba;
    uint32_t *block;
    uint8_t  *status;
} spr_request;

typedef struct {
    int64_t id;
    int32_t status;             /* SPR_OK or the render's error                 */
    int32_t passes;             /* passes of its render                         */
    int32_t batch;              /* requests in its render                       */
    int32_t reserved;
    double  t_arrival, t_admit, t_first_pass, t_done;  /* spr_server_clock     */
    int64_t blocks_decoded;     /* of its render (shared by the batch)          */
    int64_t entries;            /* ray-block entries of its render              */
    float   ms_device;          /* device time of its render                    */
} spr_result;

typedef struct {
    int64_t pending, in_flight, renderers;
    size_t  memory_used;        /* device bytes of the pooled renderers         */
    int64_t renders, requests_done, renderers_created, renderers_destroyed;
} spr_server_stats;

int spr_server_create(const spr_server_desc *desc, spr_server **out);
/* waits for the renders in flight, then releases every pooled renderer */
int spr_server_destroy(spr_server *s);
/* Register a resident volume (it must outlive the server);
 * cache_bytes_per_view (>= 8 slots) sizes the block cache of its renders:
 * a render of n views gets n times that. */
int spr_server_add_volume(spr_server *s, spr_volume *vol, size_t cache_bytes_per_view,
                          int32_t *volume_id);
/* Create an idle pooled renderer for requests of (volume, width x height)
 * batched up to n_views (<= max_batch), so that the first such request does
 * not wait for the allocation; SPR_ERR_OUT_OF_MEMORY when it does not fit
 * the budget beside the renderers already pooled.  Its graphs are captured at
 * its first render. */
int spr_server_reserve(spr_server *s, int32_t volume, int32_t width, int32_t height, int32_t n_views);
/* seconds since the server was created (a monotonic clock) */
double spr_server_clock(const spr_server *s);
/* Queue a request (copied); *id (may be NULL) numbers requests 0, 1, ... */
int spr_server_submit(spr_server *s, const spr_request *req, int64_t *id);
/* Never blocks: notes first passes, completes finished renders, admits
 * queued requests, and returns up to max_out completed requests' results in
 * completion order (*n_out of them).  A request that can never fit the
 * budget completes with SPR_ERR_OUT_OF_MEMORY. */
int spr_server_poll(spr_server *s, spr_result *out, int max_out, int *n_out);
int spr_server_info(const spr_server *s, spr_server_stats *out);

/* ---------------------------------------------------- learned speculation */
/*
 * The paper's future work (Sec. 6) suggests choosing the speculation count
 * per ray.  SPR_SPEC_LEARNED takes it from a small perceptron: 12 features
 * of each live ray at the start of a pass (pass index / 8; the current
 * block's position in the block grid, 3; the unit ray direction, 3; the
 * distance from the eye to the current block's centre over the volume
 * diagonal; the occupied fraction of its coarse cell's blocks and of its
 * super cell's coarse cells; the isovalue; the fraction of rays still live)
 * -> 64 -> 64 (ReLU) -> 2 outputs: y0 = the predicted log2 of the visible
 * blocks the ray still needs (up to and including its hit block), y1 = an
 * upper quantile of it (trained as the tau-quantile).  The ray's count is
 * min(ceil(2^(y1 + margin)), 32), capped at min(k_max, the attempt's cap);
 * with SPR_POLICY_FLOOR it is never below the paper's uniform count
 * min(k_max, floor(w*h / N_Act)): no ray then advances less per pass than
 * under the plain rule, so a learned render never takes more passes than
 * the plain one (without cache overflow), and the policy decides how much
 * further each ray speculates.  Inference runs on the
 * tensor cores (tcgen05.mma, bf16 weights and activations, fp32
 * accumulation, 128 rays per tile).  The image does not depend on the
 * policy.
 *
 * Parameters: SPR_POLICY_PARAMS floats, row-major PyTorch Linear layout:
 * W1[64][12], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
 */
#define SPR_POLICY_FEATURES 12
#define SPR_POLICY_PARAMS 5122

#define SPR_POLICY_FLOOR 1             /* counts never below the paper's uniform count */
#define SPR_POLICY_FLOOR_AFTER_FIRST 2 /* the floor from the second pass on: the first
                                        * pass takes the policy's counts alone */

/* host parameters (copied), margin and flags (0 or one of the floors);
 * synchronises the device */
int spr_set_policy(spr_renderer *r, const float *params, float margin, int flags);

/* Training traces.  While set, every pass records, for the live rays whose
 * id hashes to 0 mod sample_mod, a sample: features[12] (fp32, as the policy
 * sees them), the ray id and the visible blocks the ray took in earlier
 * passes, appended to the caller's device buffers (capacity samples; later
 * ones are dropped).  features = NULL turns tracing off.  Restarts the
 * render. */
int spr_set_trace(spr_renderer *r, float *features, uint32_t *rays, uint32_t *consumed,
                  int64_t capacity, uint32_t sample_mod);
/* After a converged render: label the samples recorded since the previous
 * call (or spr_set_trace) -- the visible blocks the ray still needed at the
 * sample, at least 1 -- into labels[i] (device, same indexing as the
 * samples); *n_samples = samples recorded so far.  Synchronises `stream`. */
int spr_trace_labels(spr_renderer *r, uint32_t *labels, int64_t *n_samples, spr_stream stream);

/* The policy on n feature rows (device, n x 12 fp32) -> out (device, n x 2
 * fp32), by the renderer's tensor-core kernel.  Synchronises `stream`. */
int spr_policy_forward(const float *params, const float *features, int64_t n, float *out,
                       spr_stream stream);
/* Mean loss over n samples (device features and labels) and its gradient
 * (host, SPR_POLICY_PARAMS floats), fp32: the loss is (y0 - t)^2 +
 * pinball_tau(t - y1) with t = log2(min(label, 64)); loss[0], loss[1] (host,
 * may be NULL) receive its two terms.  Synchronises `stream`. */
int spr_policy_grad(const float *params, const float *features, const uint32_t *labels, int64_t n,
                    float tau, float *grad, double *loss, spr_stream stream);

typedef struct {
    int32_t  epochs;
    int32_t  batch;         /* samples per Adam step                          */
    float    lr, beta1, beta2, eps;
    float    tau;           /* quantile of the second output, in (0, 1)       */
    uint32_t seed;          /* sample order                                   */
} spr_train_desc;

/* Train params (host, in/out) on n samples with Adam over the loss of
 * spr_policy_grad; loss_per_epoch (host, may be NULL) receives the mean
 * first term per epoch.  Synchronises `stream`. */
int spr_policy_train(const float *features, const uint32_t *labels, int64_t n, float *params,
                     const spr_train_desc *d, float *loss_per_epoch, spr_stream stream);

/* --------------------------------------------------------------- scan */
/* Exclusive prefix sum of n uint32 values (device in/out; in == out allowed),
 * total written to *total (device, may be NULL), by a single-pass
 * decoupled-lookback scan (the prefix sums of Sec. 3.6).  Its waits on
 * predecessor tiles are bounded: a wait that gives up returns
 * SPR_ERR_DEVICE_TIMEOUT (synchronises `stream`). */
int spr_exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                           spr_stream stream);

/* Test hook for the bounded wait: like spr_exclusive_scan_u32 but tile
 * `withhold_tile` never publishes its sum, so its successors wait until the
 * limit of `spin_limit` polls and report SPR_ERR_DEVICE_TIMEOUT. */
int spr_debug_scan_withhold(const uint32_t *in, uint32_t *out, int64_t n,
                            int64_t withhold_tile, int64_t spin_limit, spr_stream stream);

/* Allocation-free variant of spr_exclusive_scan_u32 (same arguments, same
 * results, same bounded waits).  The paper has no counterpart: it exists for
 * callers that must not allocate device memory -- one recovering from an
 * out-of-memory error, one running inside an allocator hook (allocating
 * would re-enter the allocator), one on a latency-bound stream that cannot
 * let cudaMalloc/cudaFree synchronise the device.  Its look-back scratch is
 * a static device array (256 KiB + 256 B per device), so n is limited to
 * 2^26 elements; a longer n returns SPR_ERR_INVALID_ARG before any device
 * work.  Each call clears the scratch it uses on `stream` before its launch,
 * then copies the timeout flag to the host and synchronises `stream`: every
 * call blocks the host, and none may be made on a capturing stream.  The
 * first call on a device, made with that device current, resolves the
 * scratch address (cudaGetSymbolAddress) and loads the scan kernel; under
 * CUDA's lazy module loading that first call is when the runtime places the
 * library module (its code and this array) in device memory, so make it
 * early -- before memory can run out -- and later calls allocate nothing.
 * Calls that overlap on one device (different streams or unordered host
 * threads) share the scratch and race: order them. */
int spr_exclusive_scan_u32_noalloc(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                                   spr_stream stream);

#ifdef __cplusplus
}
#endif
#endif
