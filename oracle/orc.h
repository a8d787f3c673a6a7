/*
 * orc.h -- the CPU oracle for speculative progressive isosurface raycasting
 * (Usher, Dyken, Kumar, "Speculative Progressive Raycasting for Memory
 * Constrained Isosurface Visualization of Massive Volumes", arXiv 2309.10212).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the test-suite, the smoke check and the CPU
 * baseline of the benchmark do.  It shares no source with the CUDA path.
 *
 * The oracle is written to be read against the paper, not to be fast:
 * plain loops, double precision where the geometry needs it, exact
 * predicates for every traversal decision.
 *
 * Contents
 *   1. FRC4, the fixed-rate 4^3 block transform codec that stands in for the
 *      paper's ZFP fixed-rate mode (Sec. 3.1 and 3.5: blocks of 4^3 values,
 *      each compressed to a fixed number of bits, so block b lives at a
 *      fixed byte offset and decompresses on its own).
 *   2. Value ranges of the fine (block) and coarse (4^3 blocks) macrocell
 *      grids, each combined with its +x/+y/+z neighbours (Sec. 3.1).
 *   3. Rays (Sec. 3.2, one ray per pixel), exact cell/block traversal in the
 *      manner of Amanatides and Woo (Sec. 3.3, 3.7), the ray-trilinear
 *      isosurface intersection (Sec. 3.7, after Marmitt et al.) and the
 *      per-pixel first hit (Sec. 4.4).
 *   4. The progressive pass simulator with speculation (Sec. 4): per-pass
 *      speculation count N_Spec = floor(w*h / N_Act) capped at 64, the LRU
 *      cache, and the counters of Table 2.
 */
#ifndef ORC_H
#define ORC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* 1. FRC4 codec                                                       */
/* ------------------------------------------------------------------ */
/*
 * A block holds 64 values, index i = x + 4*y + 16*z.  At rate R bits/value
 * (1 <= R <= 32) a block is exactly 64*R bits = 8*R bytes; block b of the
 * volume (x-fastest over the ceil(D/4) block grid) starts at byte 8*R*b.
 * Bit k of a block's stream is bit (k & 7) of byte (k >> 3).
 *
 * Encoding of one block (the paper uses ZFP's fixed-rate mode; this codec
 * follows the same published recipe -- common exponent, integer
 * decorrelating transform, coefficient ordering by sequency, negabinary,
 * embedded bit planes truncated at the fixed budget -- with its own choices
 * for each step):
 *   - all values zero: one 0 bit, then zero padding;
 *   - else a 1 bit and 8 bits of (emax + 127), emax = max frexp exponent of
 *     the block's nonzero values, clamped to >= -100;
 *   - q_i = round-half-even(x_i * 2^(24 - emax)), |q_i| <= 2^24;
 *   - along x, then y, then z, each 4-vector (a0,a1,a2,a3) becomes
 *     (ss, dd, d0, d1) with d0 = a1-a0, s0 = a0 + (d0>>1), d1 = a3-a2,
 *     s1 = a2 + (d1>>1), dd = s1-s0, ss = s0 + (dd>>1)  (>> is floor);
 *   - coefficients are ordered by (level(x)+level(y)+level(z), z, y, x),
 *     level = {0,1,2,2} for the four positions;
 *   - each is mapped to negabinary, u = (c + 0xAAAAAAAA) ^ 0xAAAAAAAA;
 *   - bit planes 29..0 are emitted with a remaining budget of 64R-9 bits:
 *     first the plane bit of every coefficient that is already significant
 *     (a prefix of length n), then group tests: a 1 bit if any of the
 *     remaining coefficients n..63 has this plane bit set, followed by the
 *     plane bits of coefficients n, n+1, ... up to and including the first
 *     1 (each such coefficient joins the significant prefix), repeated until
 *     a group test emits 0 or n = 64.  Emission stops the moment the budget
 *     is spent.
 * Decoding mirrors this exactly; missing bits are zero; the value is
 * (float)c_i * 2^(emax-24) (int->float round-to-nearest-even, exact scale).
 */
#define ORC_PLANES 30

int  orc_encode_block(const float in[64], int rate, uint8_t *out);
int  orc_decode_block(const uint8_t *in, int rate, float out[64]);
/* decode a block but also report the integer coefficients before the inverse
 * transform (ordered) and emax; used by the tests */
int  orc_decode_block_ints(const uint8_t *in, int rate, int32_t coeff[64], int *emax,
                           int *nonzero);

void     orc_coeff_order(int perm[64]);          /* perm[k] = block index of k-th coeff */
uint32_t orc_int_to_negabinary(int32_t x);
int32_t  orc_negabinary_to_int(uint32_t u);
void     orc_fwd_lift4(int32_t v[4]);
void     orc_inv_lift4(int32_t v[4]);
void     orc_fwd_xform(int32_t c[64]);
void     orc_inv_xform(int32_t c[64]);

/* Volume level: vol is dims[0]*dims[1]*dims[2] values, x fastest.  Partial
 * blocks at the upper faces are padded by repeating the last voxel along each
 * axis.  u8 sources are converted to float as (float)u / 255.0f. */
int orc_encode_volume_f32(const float *vol, const int32_t dims[3], int rate, uint8_t *out);
int orc_encode_volume_u8(const uint8_t *vol, const int32_t dims[3], int rate, uint8_t *out);
/* decode every block; writes only in-domain voxels, x fastest */
int orc_decode_volume(const uint8_t *comp, const int32_t dims[3], int rate, float *out);

/* ------------------------------------------------------------------ */
/* 2. Macrocell grid value ranges                                      */
/* ------------------------------------------------------------------ */
/*
 * nb[a] = ceil(D[a]/4) blocks, nc[a] = ceil(nb[a]/4) coarse cells.
 * raw(b)    = [min, max] of the decoded in-domain voxels of block b;
 * fine(b)   = union of raw(b + o), o in {0,1}^3, over neighbours that exist;
 * craw(c)   = union of raw(b) over the 4^3 blocks b of coarse cell c;
 * coarse(c) = union of craw(c + o), o in {0,1}^3, over neighbours that exist.
 * Ranges are stored as (min, max) float pairs.  iso is inside a range when
 * min <= iso <= max.
 */
int orc_ranges(const float *decoded, const int32_t dims[3],
               float *raw /* nb*2 or NULL */, float *fine /* nb*2 */,
               float *coarse /* nc*2 */);

/* ------------------------------------------------------------------ */
/* 3. Rays, traversal, intersection                                    */
/* ------------------------------------------------------------------ */
/*
 * Camera: four float triples.  The ray of pixel (i, j) (j = 0 is the bottom
 * row, linear pixel id i + W*j) starts at eye and has direction
 *     d = (p00 + (i+0.5f)*du) + (j+0.5f)*dv
 * evaluated per component in IEEE single precision, round to nearest, in
 * exactly this order and without fused multiply-add.  Points are
 * p(t) = eye + t*d, t >= 0; depth is t*|d| (voxel units).
 * Preconditions (checked): every eye component is a multiple of 2^-8 with
 * magnitude below 2^15; every volume extent is in [2, 4096].  With these, the
 * plane offsets X - eye_a (X an integer plane coordinate) are exact in single
 * precision and their products with direction components are exact in
 * double precision, so every traversal decision below is exact.
 *
 * Geometry: voxel (x,y,z) sits at point (x,y,z); the domain is
 * [0,Dx-1]x[0,Dy-1]x[0,Dz-1]; cell (x,y,z), 0 <= x <= Dx-2 etc., is the unit
 * cube with that lower corner, and the field inside is the trilinear
 * interpolant of its 8 corner voxels.  Block (bx,by,bz) owns the cells with
 * x in [4bx, 4bx+3] (likewise y, z).
 *
 * The ray visits the cells that contain p(t+) (the right limit) for t in
 * [t_enter, t_exit), in order; when it crosses several cell planes at the
 * same t it moves across all of them at once.  The first hit is the smallest
 * t at which the interpolant of the first visited cell that has a root
 * equals iso.  A block is visible to the ray when the ray visits one of its
 * cells and iso lies in fine(block); visible blocks are listed in visiting
 * order (Sec. 3.3, 4.1).
 */
typedef struct {
    int32_t dims[3];
    const float *vals;   /* dense decoded volume (x fastest), or NULL (below) */
    const float *fine;   /* fine ranges (nb*2), needed for visible-block lists */
    /* On-demand form, used when vals is NULL (Sec. 3.5: the renderer
     * decompresses the blocks its rays reach, not the whole volume).  A
     * voxel's value is read from its block, decoded from comp (FRC4 at
     * `rate`) the first time it is needed and kept in a bounded memo
     * (ORC_MEMO_LINES blocks per thread, one memo per render call).
     * Decoding is a pure function of the block's bits, so the results are
     * identical to the dense form's.  With lazy_fine and fine == NULL, the
     * fine range of a block is formed on demand from the raw ranges of its
     * +x/+y/+z neighbours (the definition of orc_ranges), so that visible
     * lists need no precomputed grid either. */
    const uint8_t *comp;
    int32_t rate;
    int32_t lazy_fine;
    int64_t *decodes;    /* if non-NULL, receives the blocks decoded by the call */
} orc_volume;

#define ORC_MEMO_LINES (1 << 16)

typedef struct {
    float eye[3], p00[3], du[3], dv[3];
} orc_camera;

/* ambiguity flags: pixels where a correct single-precision implementation may
 * legitimately differ from this oracle */
#define ORC_AMB_FACE     1u  /* hit within 1e-5 voxels of a cell face           */
#define ORC_AMB_VALUE    2u  /* |f| < 1e-5 at a cell-face crossing before the hit */
#define ORC_AMB_TANGENT  4u  /* |f| < 1e-5 at a local extremum before the hit   */
#define ORC_AMB_SHALLOW  8u  /* |df/ds| < 1e-3 per voxel of path at the hit     */

typedef struct {
    int32_t  hit;         /* 1 hit, 0 miss (also for rays that miss the box)   */
    int32_t  enters;      /* 1 when the ray enters the domain                  */
    double   t;           /* ray parameter of the hit                          */
    double   depth;       /* t*|d|                                             */
    int32_t  cell[3];     /* hit cell                                          */
    uint32_t block;       /* hit block, linear id over the nb grid, or ~0u     */
    int32_t  grey;        /* round(255*(0.1+0.9*|n.d/|d||))                     */
    uint32_t amb;         /* ORC_AMB_* flags                                   */
    int32_t  n_visible;   /* visible blocks up to and including the hit block  */
    int32_t  hit_index;   /* index of the hit block in that list, or -1        */
} orc_pixel;

int orc_check_camera(const orc_camera *cam, const int32_t dims[3]);
void orc_ray_dir(const orc_camera *cam, int W, int H, int px, int py, float d[3]);

/* Render a list of pixels (pixels == NULL: all W*H pixels in order).  With
 * full_lists the walk continues past the hit to the domain exit, so that
 * n_visible counts every visible block of the ray (the speculative traversal
 * of Sec. 4.1 may take blocks beyond the hit); otherwise it stops at the hit.
 * If vis_out is non-NULL, pixel k's visible blocks are written at
 * vis_out + vis_off[k] (offsets from the n_visible of an earlier call).
 * nthreads <= 1 runs serially. */
int orc_render(const orc_volume *vol, const orc_camera *cam, int W, int H, float iso,
               const int64_t *pixels, int64_t npix, int full_lists, orc_pixel *out,
               const int64_t *vis_off, uint32_t *vis_out, int nthreads);

/* the visited cells of one ray, in order (for tests); returns the count and
 * writes at most cap triples */
int64_t orc_trace_cells(const int32_t dims[3], const orc_camera *cam, int W, int H,
                        int px, int py, int32_t *cells, int64_t cap);

/* the right-limit block of a ray where it enters the domain (or ~0u) */
uint32_t orc_entry_block(const int32_t dims[3], const orc_camera *cam, int W, int H,
                         int px, int py);

/* Independent check: march each pixel's ray with step 1e-3 voxels, evaluate
 * the interpolant of the cell containing the sample, and bisect the first
 * sign change.  hit/t/depth only. */
int orc_march(const orc_volume *vol, const orc_camera *cam, int W, int H, float iso,
              const int64_t *pixels, int64_t npix, orc_pixel *out, int nthreads);

/* ------------------------------------------------------------------ */
/* 4. Progressive pass simulator (Sec. 3, 4)                           */
/* ------------------------------------------------------------------ */
#define ORC_SPEC_FIXED    0
#define ORC_SPEC_ADAPTIVE 1
#define ORC_SPEC_PER_RAY  2   /* each ray's own count per pass, from a table */

typedef struct {
    int32_t  pass;
    int64_t  n_active;      /* live rays at pass start (N_Act)                 */
    int32_t  k;             /* speculation count requested by the rule         */
    int32_t  k_used;        /* after overflow halving                          */
    int64_t  n_processed;   /* live rays taken this pass                       */
    int32_t  retries;       /* overflow retries                                */
    int64_t  n_entries;     /* non-empty ray-block entries                     */
    int64_t  n_visible;     /* unique visible blocks                           */
    int64_t  n_requested;   /* unique visible blocks plus +x/y/z neighbours    */
    int64_t  n_decoded;     /* cache misses = blocks decompressed              */
    int64_t  n_evicted;     /* misses that replaced a cached block             */
    int64_t  n_term_hit;    /* rays finished with a hit                        */
    int64_t  n_term_miss;   /* rays that left the volume                       */
} orc_pass_stats;

/* Simulate a render from a cold cache.  Per pixel p (all W*H pixels): enters[p],
 * hit_index[p] (-1: no hit) and its visible list vis + vis_off[p] of length
 * n_vis[p].  Returns the number of passes, or -1 on error. */
int orc_simulate(int W, int H, const int32_t dims[3],
                 const int32_t *enters, const int32_t *hit_index,
                 const int64_t *vis_off, const int32_t *n_vis, const uint32_t *vis,
                 int spec_mode, int k, int k_max, int64_t n_slots, int max_passes,
                 const int32_t *kray /* ORC_SPEC_PER_RAY: [max_passes][W*H] counts, else NULL */,
                 orc_pass_stats *stats /* max_passes */, int32_t *final_pass /* W*H or NULL */);

/* speculation count of Sec. 4: min(k_max, floor(slots / n_active)), at least 1 */
int orc_spec_count(int64_t slots, int64_t n_active, int k_max);

int orc_sizeof_pixel(void);
int orc_sizeof_pass_stats(void);
int orc_sizeof_volume(void);

#ifdef __cplusplus
}
#endif
#endif
