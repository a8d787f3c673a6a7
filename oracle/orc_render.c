/*
 * orc_render.c -- per-pixel first hit of the ray with the trilinear isosurface.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * The progressive, speculative, cached wavefront of the paper (Sec. 3, 4) is a
 * reordering of one plain computation: for each pixel, the first point along
 * its ray where the trilinear interpolant of the decoded volume equals the
 * isovalue.  This file computes exactly that, one pixel at a time:
 *   - the ray of Sec. 3.2 (eye + t*d, d formed from the camera basis);
 *   - the cells it crosses, in order, by an Amanatides-Woo walk (Sec. 3.3,
 *     3.7) whose every step is an exact comparison of crossing times;
 *   - in each crossed cell, the cubic f(s) = trilinear(u0 + s*d) - iso of
 *     Sec. 3.7 (after Marmitt et al.): split at the roots of f' into
 *     monotone pieces, take the first piece that starts on a zero or changes
 *     sign, bisect it in double precision;
 *   - the list of visible blocks in crossing order (Sec. 3.3, 4.1), i.e. the
 *     blocks whose fine range contains iso.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EPS_FACE  1e-5
#define EPS_VALUE 1e-5
#define EPS_SLOPE 1e-3
/* internal consistency flag: the hit block was not in the visible list */
#define ORC_INTERNAL_HIT_NOT_VISIBLE 0x10000u

/* a ray parameter t = n / d with d > 0.  Every n used below is an integer
 * plane coordinate minus an eye component (a multiple of 2^-8 below 2^16 in
 * magnitude: at most 24 significant bits) and every d is a direction
 * component (24 bits), so n1*d2 is exact in double and the comparison is
 * exact. */
typedef struct { double n, d; } ratio;

static int ratio_cmp(ratio a, ratio b)
{
    double l = a.n * b.d, r = b.n * a.d;
    return (l > r) - (l < r);
}

typedef struct {
    double e[3], d[3], ad[3];
    int sgn[3];
    int32_t D[3];
} ray_t;

int orc_check_camera(const orc_camera *cam, const int32_t dims[3])
{
    for (int a = 0; a < 3; a++)
        if (dims[a] < 2 || dims[a] > 4096) return -1;
    for (int a = 0; a < 3; a++) {
        double e = cam->eye[a];
        if (!isfinite(e) || fabs(e) >= 32768.0) return -2;
        if (e * 256.0 != floor(e * 256.0)) return -3;
        if (!isfinite(cam->p00[a]) || !isfinite(cam->du[a]) || !isfinite(cam->dv[a])) return -4;
    }
    return 0;
}

void orc_ray_dir(const orc_camera *cam, int W, int H, int px, int py, float d[3])
{
    (void)W;
    (void)H;
    float fi = (float)px + 0.5f;
    float fj = (float)py + 0.5f;
    for (int a = 0; a < 3; a++) {
        float t1 = fi * cam->du[a];
        float t2 = cam->p00[a] + t1;
        float t3 = fj * cam->dv[a];
        d[a] = t2 + t3;
    }
}

static void make_ray(ray_t *r, const orc_camera *cam, const int32_t dims[3], int W, int H,
                     int px, int py)
{
    float d[3];
    orc_ray_dir(cam, W, H, px, py, d);
    for (int a = 0; a < 3; a++) {
        r->e[a] = cam->eye[a];
        r->d[a] = d[a];
        r->ad[a] = fabs((double)d[a]);
        r->sgn[a] = (d[a] > 0.0f) - (d[a] < 0.0f);
        r->D[a] = dims[a];
    }
}

/* crossing time of the plane {x_a = X} */
static ratio plane_t(const ray_t *r, int a, double X)
{
    ratio t = { (X - r->e[a]) * r->sgn[a], r->ad[a] };
    return t;
}

/* entry and exit parameters of the domain box; 0 when the ray misses it or
 * only touches it */
static int ray_domain(const ray_t *r, ratio *tin, ratio *tout)
{
    ratio in = { 0.0, 1.0 }, out = { 0.0, 1.0 };
    int have_out = 0;
    for (int a = 0; a < 3; a++) {
        if (r->sgn[a] == 0) {
            if (r->e[a] < 0.0 || r->e[a] > r->D[a] - 1) return 0;
            continue;
        }
        double nearp = r->sgn[a] > 0 ? 0.0 : r->D[a] - 1;
        double farp = r->sgn[a] > 0 ? r->D[a] - 1 : 0.0;
        ratio tn = plane_t(r, a, nearp), tf = plane_t(r, a, farp);
        if (ratio_cmp(tn, in) > 0) in = tn;
        if (!have_out || ratio_cmp(tf, out) < 0) {
            out = tf;
            have_out = 1;
        }
    }
    if (!have_out) return 0;
    if (ratio_cmp(in, out) >= 0) return 0;
    *tin = in;
    *tout = out;
    return 1;
}

/* Index along axis a of the level-s cell (s = 1: cells, s = 4: blocks) that
 * contains p(T+); n cells at that level, interior planes at s*m, m = 1..n-1.
 * A floating-point estimate is corrected with exact plane tests. */
static int64_t locate(const ray_t *r, int a, ratio T, int s, int64_t n)
{
    int64_t c;
    if (r->sgn[a] == 0) {
        c = (int64_t)floor(r->e[a] / s);
        if (c < 0) c = 0;
        if (c > n - 1) c = n - 1;
        return c;
    }
    double p = r->e[a] + (T.n / T.d) * r->d[a];
    if (r->sgn[a] > 0) {
        c = (int64_t)floor(p / s);
        if (c < 0) c = 0;
        if (c > n - 1) c = n - 1;
        while (c + 1 <= n - 1 && ratio_cmp(plane_t(r, a, (double)s * (c + 1)), T) <= 0) c++;
        while (c >= 1 && ratio_cmp(plane_t(r, a, (double)s * c), T) > 0) c--;
    } else {
        c = (int64_t)ceil(p / s) - 1;
        if (c < 0) c = 0;
        if (c > n - 1) c = n - 1;
        while (c >= 1 && ratio_cmp(plane_t(r, a, (double)s * c), T) <= 0) c--;
        while (c + 1 <= n - 1 && ratio_cmp(plane_t(r, a, (double)s * (c + 1)), T) > 0) c++;
    }
    return c;
}

/* ---------------- the trilinear field in one cell ------------------------- */
/* corner k = i + 2j + 4l holds the voxel at cell + (i, j, l) */
static double tri_eval(const double v[8], const double u[3])
{
    double x = u[0], y = u[1], z = u[2];
    double c00 = v[0] * (1 - x) + v[1] * x;
    double c10 = v[2] * (1 - x) + v[3] * x;
    double c01 = v[4] * (1 - x) + v[5] * x;
    double c11 = v[6] * (1 - x) + v[7] * x;
    double c0 = c00 * (1 - y) + c10 * y;
    double c1 = c01 * (1 - y) + c11 * y;
    return c0 * (1 - z) + c1 * z;
}

static void tri_grad(const double v[8], const double u[3], double g[3])
{
    g[0] = g[1] = g[2] = 0.0;
    for (int k = 0; k < 8; k++) {
        int i = k & 1, j = (k >> 1) & 1, l = k >> 2;
        double wx = i ? u[0] : 1 - u[0], wy = j ? u[1] : 1 - u[1], wz = l ? u[2] : 1 - u[2];
        double sx = i ? 1 : -1, sy = j ? 1 : -1, sz = l ? 1 : -1;
        g[0] += v[k] * sx * wy * wz;
        g[1] += v[k] * wx * sy * wz;
        g[2] += v[k] * wx * wy * sz;
    }
}

typedef struct {
    double v[8], iso, u0[3], d[3];
    double c[4]; /* f(s) = c3 s^3 + c2 s^2 + c1 s + c0 */
} cell_fn;

static double cf_eval(const cell_fn *f, double s)
{
    double u[3] = { f->u0[0] + s * f->d[0], f->u0[1] + s * f->d[1], f->u0[2] + s * f->d[2] };
    return tri_eval(f->v, u) - f->iso;
}

static double cf_slope(const cell_fn *f, double s)
{
    return (3 * f->c[3] * s + 2 * f->c[2]) * s + f->c[1];
}

static void cf_coeffs(cell_fn *f)
{
    double c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (int k = 0; k < 8; k++) {
        int i = k & 1, j = (k >> 1) & 1, l = k >> 2;
        double ax = i ? f->u0[0] : 1 - f->u0[0], bx = i ? f->d[0] : -f->d[0];
        double ay = j ? f->u0[1] : 1 - f->u0[1], by = j ? f->d[1] : -f->d[1];
        double az = l ? f->u0[2] : 1 - f->u0[2], bz = l ? f->d[2] : -f->d[2];
        c0 += f->v[k] * ax * ay * az;
        c1 += f->v[k] * (bx * ay * az + ax * by * az + ax * ay * bz);
        c2 += f->v[k] * (bx * by * az + bx * ay * bz + ax * by * bz);
        c3 += f->v[k] * bx * by * bz;
    }
    f->c[0] = c0 - f->iso;
    f->c[1] = c1;
    f->c[2] = c2;
    f->c[3] = c3;
}

/* roots of f' strictly inside (0, L), ascending */
static int deriv_roots(const cell_fn *f, double L, double out[2])
{
    double a = 3 * f->c[3], b = 2 * f->c[2], c = f->c[1];
    double r[2];
    int n = 0;
    if (a == 0.0) {
        if (b != 0.0) r[n++] = -c / b;
    } else {
        double disc = b * b - 4 * a * c;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            double q = -0.5 * (b + (b >= 0 ? sq : -sq));
            if (q != 0.0) {
                r[n++] = q / a;
                r[n++] = c / q;
            } else {
                r[n++] = 0.0;
            }
        }
    }
    int m = 0;
    for (int i = 0; i < n; i++)
        if (r[i] > 0.0 && r[i] < L) out[m++] = r[i];
    if (m == 2) {
        if (out[0] > out[1]) {
            double t = out[0];
            out[0] = out[1];
            out[1] = t;
        }
        if (out[0] == out[1]) m = 1;
    }
    return m;
}

/* First root of f in [0, L]; flags small |f| at the points examined before it. */
static int cell_first_root(const cell_fn *f, double L, double *s_hit, uint32_t *amb)
{
    double pts[4];
    int np = 0;
    double ext[2];
    int ne = deriv_roots(f, L, ext);
    pts[np++] = 0.0;
    for (int i = 0; i < ne; i++) pts[np++] = ext[i];
    pts[np++] = L;

    double fa = cf_eval(f, 0.0);
    if (fabs(fa) < EPS_VALUE) *amb |= ORC_AMB_VALUE;
    if (fa == 0.0) {
        *s_hit = 0.0;
        return 1;
    }
    for (int i = 1; i < np; i++) {
        double sa = pts[i - 1], sb = pts[i];
        double fb = cf_eval(f, sb);
        if (fb == 0.0) {
            *s_hit = sb;
            return 1;
        }
        if ((fb < 0.0) != (fa < 0.0)) {
            double lo = sa, hi = sb, flo = fa;
            for (int it = 0; it < 200 && hi - lo > 1e-14 * (1.0 + fabs(hi)); it++) {
                double mid = 0.5 * (lo + hi), fm = cf_eval(f, mid);
                if (fm == 0.0) {
                    lo = hi = mid;
                    break;
                }
                if ((fm < 0.0) == (flo < 0.0)) {
                    lo = mid;
                    flo = fm;
                } else {
                    hi = mid;
                }
            }
            *s_hit = 0.5 * (lo + hi);
            return 1;
        }
        if (fabs(fb) < EPS_VALUE) *amb |= (i < np - 1) ? ORC_AMB_TANGENT : ORC_AMB_VALUE;
        fa = fb;
    }
    return 0;
}

/* ---------------- voxel access: dense, or blocks decoded on demand ---------- */
/* One reader per thread and render call.  In the on-demand form a memo line
 * holds one decoded block (64 values, x fastest) and the min/max of its
 * in-domain voxels; line = hash(block id), replaced when another block
 * maps there. */
typedef struct {
    const orc_volume *vol;
    int64_t nb[3];
    int64_t *tag;    /* block held by each line, -1 when empty */
    float *val;      /* 64 values per line */
    float *raw;      /* min, max per line */
    int64_t decodes;
    int ok;
} orc_reader;

static int reader_init(orc_reader *rd, const orc_volume *vol)
{
    memset(rd, 0, sizeof *rd);
    rd->vol = vol;
    rd->ok = 1;
    for (int a = 0; a < 3; a++) rd->nb[a] = (vol->dims[a] + 3) / 4;
    if (vol->vals) return 0;
    if (!vol->comp || vol->rate < 1 || vol->rate > 32) return -1;
    rd->tag = (int64_t *)malloc(sizeof(int64_t) * ORC_MEMO_LINES);
    rd->val = (float *)malloc(sizeof(float) * 64 * ORC_MEMO_LINES);
    rd->raw = (float *)malloc(sizeof(float) * 2 * ORC_MEMO_LINES);
    if (!rd->tag || !rd->val || !rd->raw) return -2;
    for (int64_t i = 0; i < ORC_MEMO_LINES; i++) rd->tag[i] = -1;
    return 0;
}

static void reader_free(orc_reader *rd)
{
    free(rd->tag);
    free(rd->val);
    free(rd->raw);
    rd->tag = NULL;
    rd->val = rd->raw = NULL;
}

/* the memo line holding decoded block b (decoding it if it is not there) */
static int64_t reader_line(orc_reader *rd, int64_t b)
{
    uint64_t h = (uint64_t)b * 0x9E3779B97F4A7C15ull;
    int64_t line = (int64_t)(h >> 48) & (ORC_MEMO_LINES - 1);
    if (rd->tag[line] == b) return line;
    const orc_volume *vol = rd->vol;
    float *v = rd->val + 64 * line;
    if (orc_decode_block(vol->comp + b * 8 * (int64_t)vol->rate, vol->rate, v)) rd->ok = 0;
    rd->decodes++;
    /* min/max of the block's in-domain voxels (raw(b) of orc_ranges) */
    int64_t bx = b % rd->nb[0], by = (b / rd->nb[0]) % rd->nb[1], bz = b / (rd->nb[0] * rd->nb[1]);
    float mn = INFINITY, mx = -INFINITY;
    for (int z = 0; z < 4 && 4 * bz + z < vol->dims[2]; z++)
        for (int y = 0; y < 4 && 4 * by + y < vol->dims[1]; y++)
            for (int x = 0; x < 4 && 4 * bx + x < vol->dims[0]; x++) {
                float q = v[x + 4 * y + 16 * z];
                if (q < mn) mn = q;
                if (q > mx) mx = q;
            }
    rd->raw[2 * line] = mn;
    rd->raw[2 * line + 1] = mx;
    rd->tag[line] = b;
    return line;
}

static double voxel(orc_reader *rd, int64_t x, int64_t y, int64_t z)
{
    const orc_volume *vol = rd->vol;
    if (vol->vals) return vol->vals[x + (int64_t)vol->dims[0] * (y + (int64_t)vol->dims[1] * z)];
    int64_t b = (x >> 2) + rd->nb[0] * ((y >> 2) + rd->nb[1] * (z >> 2));
    int64_t line = reader_line(rd, b);
    return rd->val[64 * line + (x & 3) + 4 * (y & 3) + 16 * (z & 3)];
}

/* 1 when iso lies in the fine range of block b, 0 when not, -1 when the
 * volume has no fine ranges (no visible lists) */
static int block_visible(orc_reader *rd, int64_t b, float iso)
{
    const orc_volume *vol = rd->vol;
    if (vol->fine) return vol->fine[2 * b] <= iso && iso <= vol->fine[2 * b + 1];
    if (vol->vals || !vol->lazy_fine) return -1;
    /* fine(b) = union of raw(b + o), o in {0,1}^3, over neighbours that exist */
    int64_t bx = b % rd->nb[0], by = (b / rd->nb[0]) % rd->nb[1], bz = b / (rd->nb[0] * rd->nb[1]);
    float mn = INFINITY, mx = -INFINITY;
    for (int o = 0; o < 8; o++) {
        int64_t x = bx + (o & 1), y = by + ((o >> 1) & 1), z = bz + (o >> 2);
        if (x >= rd->nb[0] || y >= rd->nb[1] || z >= rd->nb[2]) continue;
        int64_t line = reader_line(rd, x + rd->nb[0] * (y + rd->nb[1] * z));
        if (rd->raw[2 * line] < mn) mn = rd->raw[2 * line];
        if (rd->raw[2 * line + 1] > mx) mx = rd->raw[2 * line + 1];
    }
    return mn <= iso && iso <= mx;
}

static void cell_corners(orc_reader *rd, const int64_t c[3], double v[8])
{
    for (int k = 0; k < 8; k++)
        v[k] = voxel(rd, c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + (k >> 2));
}

/* readers for up to n threads; returns NULL on failure */
static orc_reader *readers_new(const orc_volume *vol, int n)
{
    orc_reader *rd = (orc_reader *)calloc((size_t)n, sizeof(orc_reader));
    if (!rd) return NULL;
    for (int i = 0; i < n; i++)
        if (reader_init(&rd[i], vol)) {
            for (int j = 0; j <= i; j++) reader_free(&rd[j]);
            free(rd);
            return NULL;
        }
    return rd;
}

/* frees the readers; returns -1 if a block failed to decode */
static int readers_done(const orc_volume *vol, orc_reader *rd, int n)
{
    int64_t dec = 0;
    int ok = 1;
    for (int i = 0; i < n; i++) {
        dec += rd[i].decodes;
        ok &= rd[i].ok;
        reader_free(&rd[i]);
    }
    free(rd);
    if (vol->decodes) *vol->decodes = dec;
    return ok ? 0 : -1;
}

static int thread_index(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* ---------------- one pixel ---------------------------------------------- */
static void render_pixel(orc_reader *rd, const ray_t *r, float iso, int full_list,
                         orc_pixel *out, uint32_t *vis_out)
{
    const orc_volume *vol = rd->vol;
    memset(out, 0, sizeof *out);
    out->t = INFINITY;
    out->depth = INFINITY;
    out->cell[0] = out->cell[1] = out->cell[2] = -1;
    out->block = 0xFFFFFFFFu;
    out->hit_index = -1;

    ratio T, Tend;
    if (!ray_domain(r, &T, &Tend)) return;
    out->enters = 1;

    const int32_t *D = vol->dims;
    int64_t nb[3] = { (D[0] + 3) / 4, (D[1] + 3) / 4, (D[2] + 3) / 4 };
    int64_t c[3];
    for (int a = 0; a < 3; a++) c[a] = locate(r, a, T, 1, D[a] - 1);
    double dn = sqrt(r->d[0] * r->d[0] + r->d[1] * r->d[1] + r->d[2] * r->d[2]);
    int64_t prev_block = -1;

    for (;;) {
        /* next crossing: every axis whose next plane is crossed first */
        ratio tmin = { 0.0, 1.0 };
        int mask = 0, have = 0;
        for (int a = 0; a < 3; a++) {
            if (r->sgn[a] == 0) continue;
            double X = r->sgn[a] > 0 ? (double)(c[a] + 1) : (double)c[a];
            ratio ta = plane_t(r, a, X);
            int cmp = have ? ratio_cmp(ta, tmin) : -1;
            if (cmp < 0) {
                tmin = ta;
                mask = 1 << a;
                have = 1;
            } else if (cmp == 0) {
                mask |= 1 << a;
            }
        }

        int64_t bid = (c[0] >> 2) + nb[0] * ((c[1] >> 2) + nb[1] * (c[2] >> 2));
        if (bid != prev_block) {
            prev_block = bid;
            if (block_visible(rd, bid, iso) == 1) {
                if (vis_out) vis_out[out->n_visible] = (uint32_t)bid;
                out->n_visible++;
            }
        }

        if (!out->hit) {
            cell_fn f;
            cell_corners(rd, c, f.v);
            int below = 0, above = 0;
            for (int k = 0; k < 8; k++) {
                below += f.v[k] < iso;
                above += f.v[k] > iso;
            }
            if (below != 8 && above != 8) {
                double t0 = T.n / T.d, t1 = tmin.n / tmin.d;
                f.iso = iso;
                for (int a = 0; a < 3; a++) {
                    f.d[a] = r->d[a];
                    f.u0[a] = (r->e[a] - (double)c[a]) + t0 * r->d[a];
                }
                cf_coeffs(&f);
                double s;
                if (cell_first_root(&f, t1 - t0, &s, &out->amb)) {
                    out->hit = 1;
                    out->t = t0 + s;
                    out->depth = out->t * dn;
                    for (int a = 0; a < 3; a++) out->cell[a] = (int32_t)c[a];
                    out->block = (uint32_t)bid;
                    out->hit_index = out->n_visible - 1;
                    if (block_visible(rd, bid, iso) == 0) out->amb |= ORC_INTERNAL_HIT_NOT_VISIBLE;
                    for (int a = 0; a < 3; a++) {
                        double p = r->e[a] + out->t * r->d[a];
                        if (fabs(p - rint(p)) < EPS_FACE) out->amb |= ORC_AMB_FACE;
                    }
                    if (fabs(cf_slope(&f, s)) / dn < EPS_SLOPE) out->amb |= ORC_AMB_SHALLOW;
                    double u[3] = { f.u0[0] + s * f.d[0], f.u0[1] + s * f.d[1],
                                    f.u0[2] + s * f.d[2] };
                    double g[3];
                    tri_grad(f.v, u, g);
                    double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                    double cosv = gn > 0.0
                        ? fabs(g[0] * r->d[0] + g[1] * r->d[1] + g[2] * r->d[2]) / (gn * dn)
                        : 0.0;
                    out->grey = (int32_t)floor(255.0 * (0.1 + 0.9 * cosv) + 0.5);
                    if (!full_list) return;
                }
            }
        }

        int leaves = 0;
        for (int a = 0; a < 3; a++) {
            if (!(mask >> a & 1)) continue;
            c[a] += r->sgn[a];
            if (c[a] < 0 || c[a] > D[a] - 2) leaves = 1;
        }
        if (leaves) break;
        T = tmin;
    }
}

int orc_render(const orc_volume *vol, const orc_camera *cam, int W, int H, float iso,
               const int64_t *pixels, int64_t npix, int full_lists, orc_pixel *out,
               const int64_t *vis_off, uint32_t *vis_out, int nthreads)
{
    if (orc_check_camera(cam, vol->dims)) return -1;
    if (W < 1 || H < 1) return -1;
    if (!pixels) npix = (int64_t)W * H;
    if (nthreads < 1) nthreads = 1;
#ifndef _OPENMP
    nthreads = 1;
#endif
    orc_reader *rd = readers_new(vol, nthreads);
    if (!rd) return -2;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t k = 0; k < npix; k++) {
        int64_t p = pixels ? pixels[k] : k;
        ray_t r;
        make_ray(&r, cam, vol->dims, W, H, (int)(p % W), (int)(p / W));
        render_pixel(&rd[thread_index()], &r, iso, full_lists, &out[k],
                     (vis_off && vis_out) ? vis_out + vis_off[k] : NULL);
    }
    return readers_done(vol, rd, nthreads) ? -3 : 0;
}

int64_t orc_trace_cells(const int32_t dims[3], const orc_camera *cam, int W, int H, int px,
                        int py, int32_t *cells, int64_t cap)
{
    ray_t r;
    make_ray(&r, cam, dims, W, H, px, py);
    ratio T, Tend;
    if (!ray_domain(&r, &T, &Tend)) return 0;
    int64_t c[3], n = 0;
    for (int a = 0; a < 3; a++) c[a] = locate(&r, a, T, 1, dims[a] - 1);
    for (;;) {
        if (n < cap) {
            cells[3 * n] = (int32_t)c[0];
            cells[3 * n + 1] = (int32_t)c[1];
            cells[3 * n + 2] = (int32_t)c[2];
        }
        n++;
        ratio tmin = { 0.0, 1.0 };
        int mask = 0, have = 0;
        for (int a = 0; a < 3; a++) {
            if (r.sgn[a] == 0) continue;
            double X = r.sgn[a] > 0 ? (double)(c[a] + 1) : (double)c[a];
            ratio ta = plane_t(&r, a, X);
            int cmp = have ? ratio_cmp(ta, tmin) : -1;
            if (cmp < 0) {
                tmin = ta;
                mask = 1 << a;
                have = 1;
            } else if (cmp == 0) {
                mask |= 1 << a;
            }
        }
        int leaves = 0;
        for (int a = 0; a < 3; a++) {
            if (!(mask >> a & 1)) continue;
            c[a] += r.sgn[a];
            if (c[a] < 0 || c[a] > dims[a] - 2) leaves = 1;
        }
        if (leaves) break;
        T = tmin;
    }
    return n;
}

uint32_t orc_entry_block(const int32_t dims[3], const orc_camera *cam, int W, int H, int px,
                         int py)
{
    ray_t r;
    make_ray(&r, cam, dims, W, H, px, py);
    ratio T, Tend;
    if (!ray_domain(&r, &T, &Tend)) return 0xFFFFFFFFu;
    int64_t nb[3] = { (dims[0] + 3) / 4, (dims[1] + 3) / 4, (dims[2] + 3) / 4 };
    int64_t c[3];
    for (int a = 0; a < 3; a++) c[a] = locate(&r, a, T, 1, dims[a] - 1);
    return (uint32_t)((c[0] >> 2) + nb[0] * ((c[1] >> 2) + nb[1] * (c[2] >> 2)));
}

/* ---------------- independent dense march --------------------------------- */
static double field_at(orc_reader *rd, const double p[3], double iso)
{
    const orc_volume *vol = rd->vol;
    int64_t c[3];
    double u[3], v[8];
    for (int a = 0; a < 3; a++) {
        double f = floor(p[a]);
        if (f < 0) f = 0;
        if (f > vol->dims[a] - 2) f = vol->dims[a] - 2;
        c[a] = (int64_t)f;
        u[a] = p[a] - f;
    }
    cell_corners(rd, c, v);
    return tri_eval(v, u) - iso;
}

int orc_march(const orc_volume *vol, const orc_camera *cam, int W, int H, float iso,
              const int64_t *pixels, int64_t npix, orc_pixel *out, int nthreads)
{
    if (orc_check_camera(cam, vol->dims)) return -1;
    if (!pixels) npix = (int64_t)W * H;
    if (nthreads < 1) nthreads = 1;
#ifndef _OPENMP
    nthreads = 1;
#endif
    orc_reader *rds = readers_new(vol, nthreads);
    if (!rds) return -2;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t k = 0; k < npix; k++) {
        orc_reader *rd = &rds[thread_index()];
        int64_t pix = pixels ? pixels[k] : k;
        ray_t r;
        make_ray(&r, cam, vol->dims, W, H, (int)(pix % W), (int)(pix / W));
        orc_pixel *o = &out[k];
        memset(o, 0, sizeof *o);
        o->t = INFINITY;
        o->depth = INFINITY;
        o->block = 0xFFFFFFFFu;
        o->hit_index = -1;
        o->cell[0] = o->cell[1] = o->cell[2] = -1;
        ratio T, Tend;
        if (!ray_domain(&r, &T, &Tend)) continue;
        o->enters = 1;
        double t0 = T.n / T.d, t1 = Tend.n / Tend.d;
        double dn = sqrt(r.d[0] * r.d[0] + r.d[1] * r.d[1] + r.d[2] * r.d[2]);
        double dt = 1e-3 / dn;
        double p[3];
        for (int a = 0; a < 3; a++) p[a] = r.e[a] + t0 * r.d[a];
        double tp = t0, fp = field_at(rd, p, iso);
        if (fp == 0.0) {
            o->hit = 1;
            o->t = t0;
        } else {
            for (int64_t i = 1;; i++) {
                double t = t0 + (double)i * dt;
                if (t > t1) t = t1;
                for (int a = 0; a < 3; a++) p[a] = r.e[a] + t * r.d[a];
                double f = field_at(rd, p, iso);
                if (f == 0.0 || (f < 0.0) != (fp < 0.0)) {
                    double lo = tp, hi = t, flo = fp;
                    if (f != 0.0) {
                        for (int it = 0; it < 200 && hi - lo > 1e-14 * (1.0 + fabs(hi)); it++) {
                            double mid = 0.5 * (lo + hi), q[3];
                            for (int a = 0; a < 3; a++) q[a] = r.e[a] + mid * r.d[a];
                            double fm = field_at(rd, q, iso);
                            if (fm == 0.0) {
                                lo = hi = mid;
                                break;
                            }
                            if ((fm < 0.0) == (flo < 0.0)) {
                                lo = mid;
                                flo = fm;
                            } else {
                                hi = mid;
                            }
                        }
                        o->t = 0.5 * (lo + hi);
                    } else {
                        o->t = t;
                    }
                    o->hit = 1;
                    break;
                }
                if (t >= t1) break;
                tp = t;
                fp = f;
            }
        }
        if (o->hit) o->depth = o->t * dn;
    }
    return readers_done(vol, rds, nthreads) ? -3 : 0;
}
