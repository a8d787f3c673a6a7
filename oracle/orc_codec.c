/*
 * orc_codec.c -- FRC4, the oracle's fixed-rate 4^3 block codec.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * The paper stores the volume ZFP-compressed in fixed-rate mode and
 * decompresses single blocks on demand (Sec. 3.1, 3.5).  FRC4 is this
 * project's own codec of that kind; every step is spelled out in orc.h.
 * This file is the plain, bit-at-a-time rendition of that definition.
 */
#include "orc.h"

#include <limits.h>
#include <math.h>
#include <string.h>

/* ---------------- bit I/O: bit k lives in byte k>>3 at bit k&7 ---------- */
typedef struct { uint8_t *buf; int64_t pos; } bit_writer;
typedef struct { const uint8_t *buf; int64_t pos; } bit_reader;

static void put_bit(bit_writer *w, int b)
{
    if (b) w->buf[w->pos >> 3] |= (uint8_t)(1u << (w->pos & 7));
    w->pos++;
}

static int get_bit(bit_reader *r)
{
    int b = (r->buf[r->pos >> 3] >> (r->pos & 7)) & 1;
    r->pos++;
    return b;
}

/* ---------------- the integer decorrelating transform -------------------- */
/* Additions wrap modulo 2^32 (they never do for streams the encoder writes,
 * but the decoder accepts any bits).  Arithmetic right shift of a negative
 * int is floor division by two with gcc and clang (two's complement). */
static int32_t add_w(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
static int32_t sub_w(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }

void orc_fwd_lift4(int32_t v[4])
{
    int32_t a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
    int32_t d0 = sub_w(a1, a0), s0 = add_w(a0, d0 >> 1);
    int32_t d1 = sub_w(a3, a2), s1 = add_w(a2, d1 >> 1);
    int32_t dd = sub_w(s1, s0), ss = add_w(s0, dd >> 1);
    v[0] = ss; v[1] = dd; v[2] = d0; v[3] = d1;
}

void orc_inv_lift4(int32_t v[4])
{
    int32_t ss = v[0], dd = v[1], d0 = v[2], d1 = v[3];
    int32_t s0 = sub_w(ss, dd >> 1);
    int32_t s1 = add_w(s0, dd);
    int32_t a0 = sub_w(s0, d0 >> 1);
    int32_t a1 = add_w(a0, d0);
    int32_t a2 = sub_w(s1, d1 >> 1);
    int32_t a3 = add_w(a2, d1);
    v[0] = a0; v[1] = a1; v[2] = a2; v[3] = a3;
}

/* apply a 1-D lifting step to the 16 lines along axis `axis` */
static void lift_axis(int32_t c[64], int axis, int inverse)
{
    int stride = axis == 0 ? 1 : (axis == 1 ? 4 : 16);
    for (int line = 0; line < 16; line++) {
        /* the two coordinates that are not `axis` */
        int u = line & 3, w = line >> 2, base;
        if (axis == 0)      base = 4 * u + 16 * w;
        else if (axis == 1) base = u + 16 * w;
        else                base = u + 4 * w;
        int32_t v[4];
        for (int i = 0; i < 4; i++) v[i] = c[base + i * stride];
        if (inverse) orc_inv_lift4(v); else orc_fwd_lift4(v);
        for (int i = 0; i < 4; i++) c[base + i * stride] = v[i];
    }
}

void orc_fwd_xform(int32_t c[64])
{
    lift_axis(c, 0, 0);
    lift_axis(c, 1, 0);
    lift_axis(c, 2, 0);
}

void orc_inv_xform(int32_t c[64])
{
    lift_axis(c, 2, 1);
    lift_axis(c, 1, 1);
    lift_axis(c, 0, 1);
}

/* ---------------- coefficient order ------------------------------------ */
static int level_of(int pos) { return pos == 0 ? 0 : (pos == 1 ? 1 : 2); }

void orc_coeff_order(int perm[64])
{
    int k = 0;
    for (int s = 0; s <= 6; s++)
        for (int z = 0; z < 4; z++)
            for (int y = 0; y < 4; y++)
                for (int x = 0; x < 4; x++)
                    if (level_of(x) + level_of(y) + level_of(z) == s)
                        perm[k++] = x + 4 * y + 16 * z;
}

/* ---------------- negabinary ------------------------------------------- */
uint32_t orc_int_to_negabinary(int32_t x)
{
    return ((uint32_t)x + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}

int32_t orc_negabinary_to_int(uint32_t u)
{
    return (int32_t)((u ^ 0xAAAAAAAAu) - 0xAAAAAAAAu);
}

/* ---------------- block encode / decode -------------------------------- */
int orc_encode_block(const float in[64], int rate, uint8_t *out)
{
    if (rate < 1 || rate > 32) return -1;
    int64_t maxbits = 64 * (int64_t)rate;
    memset(out, 0, (size_t)(8 * rate));
    bit_writer w = { out, 0 };

    int emax = INT_MIN;
    for (int i = 0; i < 64; i++) {
        if (!isfinite(in[i])) return -2;
        if (in[i] != 0.0f) {
            int e;
            frexp((double)in[i], &e);
            if (e > emax) emax = e;
        }
    }
    if (emax == INT_MIN) {          /* all-zero block */
        put_bit(&w, 0);
        return 0;
    }
    if (emax < -100) emax = -100;
    put_bit(&w, 1);
    for (int b = 0; b < 8; b++) put_bit(&w, ((emax + 127) >> b) & 1);

    int32_t q[64];
    for (int i = 0; i < 64; i++)
        q[i] = (int32_t)nearbyint(ldexp((double)in[i], 24 - emax));
    orc_fwd_xform(q);

    int perm[64];
    orc_coeff_order(perm);
    uint32_t u[64];
    for (int k = 0; k < 64; k++) u[k] = orc_int_to_negabinary(q[perm[k]]);

    int64_t budget = maxbits - 9;
    int n = 0;
    for (int p = ORC_PLANES - 1; p >= 0 && budget > 0; p--) {
        for (int i = 0; i < n && budget > 0; i++) {
            put_bit(&w, (u[i] >> p) & 1);
            budget--;
        }
        while (n < 64 && budget > 0) {
            int any = 0;
            for (int j = n; j < 64; j++) any |= (u[j] >> p) & 1;
            put_bit(&w, any);
            budget--;
            if (!any) break;
            while (n < 64 && budget > 0) {
                int b = (u[n] >> p) & 1;
                put_bit(&w, b);
                budget--;
                n++;
                if (b) break;
            }
        }
    }
    return 0;
}

int orc_decode_block_ints(const uint8_t *in, int rate, int32_t coeff[64], int *emax_out,
                          int *nonzero)
{
    if (rate < 1 || rate > 32) return -1;
    int64_t maxbits = 64 * (int64_t)rate;
    bit_reader r = { in, 0 };
    for (int k = 0; k < 64; k++) coeff[k] = 0;
    if (!get_bit(&r)) {
        *nonzero = 0;
        *emax_out = 0;
        return 0;
    }
    *nonzero = 1;
    int e8 = 0;
    for (int b = 0; b < 8; b++) e8 |= get_bit(&r) << b;
    int emax = e8 - 127;
    if (emax < -100) emax = -100;
    *emax_out = emax;

    uint32_t u[64] = { 0 };
    int64_t budget = maxbits - 9;
    int n = 0;
    for (int p = ORC_PLANES - 1; p >= 0 && budget > 0; p--) {
        for (int i = 0; i < n && budget > 0; i++) {
            u[i] |= (uint32_t)get_bit(&r) << p;
            budget--;
        }
        while (n < 64 && budget > 0) {
            int any = get_bit(&r);
            budget--;
            if (!any) break;
            while (n < 64 && budget > 0) {
                int b = get_bit(&r);
                budget--;
                n++;
                if (b) {
                    u[n - 1] |= 1u << p;
                    break;
                }
            }
        }
    }
    for (int k = 0; k < 64; k++) coeff[k] = orc_negabinary_to_int(u[k]);
    return 0;
}

int orc_decode_block(const uint8_t *in, int rate, float out[64])
{
    int32_t ordered[64], c[64];
    int emax, nonzero;
    int rc = orc_decode_block_ints(in, rate, ordered, &emax, &nonzero);
    if (rc) return rc;
    if (!nonzero) {
        for (int i = 0; i < 64; i++) out[i] = 0.0f;
        return 0;
    }
    int perm[64];
    orc_coeff_order(perm);
    for (int k = 0; k < 64; k++) c[perm[k]] = ordered[k];
    orc_inv_xform(c);
    float scale = ldexpf(1.0f, emax - 24);      /* exact: emax >= -100 */
    for (int i = 0; i < 64; i++) out[i] = (float)c[i] * scale;
    return 0;
}

/* ---------------- volume level ----------------------------------------- */
static int64_t idx3(const int32_t d[3], int64_t x, int64_t y, int64_t z)
{
    return x + (int64_t)d[0] * (y + (int64_t)d[1] * z);
}

static int check_dims(const int32_t dims[3])
{
    for (int a = 0; a < 3; a++)
        if (dims[a] < 1) return -1;
    return 0;
}

static int encode_volume(const float *vf, const uint8_t *vu, const int32_t dims[3], int rate,
                         uint8_t *out)
{
    if (check_dims(dims) || rate < 1 || rate > 32) return -1;
    int64_t nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (dims[a] + 3) / 4;
    int64_t bytes = 8 * (int64_t)rate;
    int bad = 0;
    /* blocks are independent: the rows of blocks are encoded in parallel */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) collapse(2) reduction(| : bad)
#endif
    for (int64_t bz = 0; bz < nb[2]; bz++)
        for (int64_t by = 0; by < nb[1]; by++)
            for (int64_t bx = 0; bx < nb[0]; bx++) {
                float blk[64];
                for (int z = 0; z < 4; z++)
                    for (int y = 0; y < 4; y++)
                        for (int x = 0; x < 4; x++) {
                            int64_t gx = 4 * bx + x, gy = 4 * by + y, gz = 4 * bz + z;
                            if (gx > dims[0] - 1) gx = dims[0] - 1;
                            if (gy > dims[1] - 1) gy = dims[1] - 1;
                            if (gz > dims[2] - 1) gz = dims[2] - 1;
                            int64_t g = idx3(dims, gx, gy, gz);
                            blk[x + 4 * y + 16 * z] = vf ? vf[g] : (float)vu[g] / 255.0f;
                        }
                int64_t b = bx + nb[0] * (by + nb[1] * bz);
                if (orc_encode_block(blk, rate, out + b * bytes)) bad = 1;
            }
    return bad ? -1 : 0;
}

int orc_encode_volume_f32(const float *vol, const int32_t dims[3], int rate, uint8_t *out)
{
    return encode_volume(vol, NULL, dims, rate, out);
}

int orc_encode_volume_u8(const uint8_t *vol, const int32_t dims[3], int rate, uint8_t *out)
{
    return encode_volume(NULL, vol, dims, rate, out);
}

int orc_decode_volume(const uint8_t *comp, const int32_t dims[3], int rate, float *out)
{
    if (check_dims(dims) || rate < 1 || rate > 32) return -1;
    int64_t nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (dims[a] + 3) / 4;
    int64_t bytes = 8 * (int64_t)rate;
    for (int64_t bz = 0; bz < nb[2]; bz++)
        for (int64_t by = 0; by < nb[1]; by++)
            for (int64_t bx = 0; bx < nb[0]; bx++) {
                int64_t b = bx + nb[0] * (by + nb[1] * bz);
                float blk[64];
                int rc = orc_decode_block(comp + b * bytes, rate, blk);
                if (rc) return rc;
                for (int z = 0; z < 4; z++)
                    for (int y = 0; y < 4; y++)
                        for (int x = 0; x < 4; x++) {
                            int64_t gx = 4 * bx + x, gy = 4 * by + y, gz = 4 * bz + z;
                            if (gx < dims[0] && gy < dims[1] && gz < dims[2])
                                out[idx3(dims, gx, gy, gz)] = blk[x + 4 * y + 16 * z];
                        }
            }
    return 0;
}
