/*
 * orc_grid.c -- value ranges of the fine and coarse macrocell grids.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Sec. 3.1: the fine grid has one cell per 4^3 compressed block, the coarse
 * grid one cell per 4^3 blocks (16^3 voxels).  A cell's range is its own
 * range combined with the ranges of its neighbours in +x, +y and +z (faces,
 * edges and the corner), so that the dual cells straddling the +faces are
 * covered and no crack appears.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>

static void grow(float *mn, float *mx, float lo, float hi)
{
    if (lo < *mn) *mn = lo;
    if (hi > *mx) *mx = hi;
}

int orc_ranges(const float *dec, const int32_t dims[3], float *raw_out, float *fine,
               float *coarse)
{
    int64_t nb[3], nc[3];
    for (int a = 0; a < 3; a++) {
        if (dims[a] < 2) return -1;
        nb[a] = (dims[a] + 3) / 4;
        nc[a] = (nb[a] + 3) / 4;
    }
    int64_t nblocks = nb[0] * nb[1] * nb[2];
    int64_t ncells = nc[0] * nc[1] * nc[2];
    float *raw = raw_out ? raw_out : (float *)malloc(sizeof(float) * 2 * nblocks);
    float *craw = (float *)malloc(sizeof(float) * 2 * ncells);
    if (!raw || !craw) {
        if (!raw_out) free(raw);
        free(craw);
        return -2;
    }

    /* own range of each block: decoded voxels inside the domain */
    for (int64_t bz = 0; bz < nb[2]; bz++)
        for (int64_t by = 0; by < nb[1]; by++)
            for (int64_t bx = 0; bx < nb[0]; bx++) {
                float mn = INFINITY, mx = -INFINITY;
                for (int64_t z = 4 * bz; z < 4 * bz + 4 && z < dims[2]; z++)
                    for (int64_t y = 4 * by; y < 4 * by + 4 && y < dims[1]; y++)
                        for (int64_t x = 4 * bx; x < 4 * bx + 4 && x < dims[0]; x++) {
                            float v = dec[x + dims[0] * (y + dims[1] * z)];
                            grow(&mn, &mx, v, v);
                        }
                int64_t b = bx + nb[0] * (by + nb[1] * bz);
                raw[2 * b] = mn;
                raw[2 * b + 1] = mx;
            }

    /* fine: own range with the +x/+y/+z face, edge and corner neighbours */
    for (int64_t bz = 0; bz < nb[2]; bz++)
        for (int64_t by = 0; by < nb[1]; by++)
            for (int64_t bx = 0; bx < nb[0]; bx++) {
                float mn = INFINITY, mx = -INFINITY;
                for (int o = 0; o < 8; o++) {
                    int64_t x = bx + (o & 1), y = by + ((o >> 1) & 1), z = bz + (o >> 2);
                    if (x >= nb[0] || y >= nb[1] || z >= nb[2]) continue;
                    int64_t n = x + nb[0] * (y + nb[1] * z);
                    grow(&mn, &mx, raw[2 * n], raw[2 * n + 1]);
                }
                int64_t b = bx + nb[0] * (by + nb[1] * bz);
                fine[2 * b] = mn;
                fine[2 * b + 1] = mx;
            }

    /* coarse: range of the 4^3 blocks of each coarse cell ... */
    for (int64_t cz = 0; cz < nc[2]; cz++)
        for (int64_t cy = 0; cy < nc[1]; cy++)
            for (int64_t cx = 0; cx < nc[0]; cx++) {
                float mn = INFINITY, mx = -INFINITY;
                for (int64_t z = 4 * cz; z < 4 * cz + 4 && z < nb[2]; z++)
                    for (int64_t y = 4 * cy; y < 4 * cy + 4 && y < nb[1]; y++)
                        for (int64_t x = 4 * cx; x < 4 * cx + 4 && x < nb[0]; x++) {
                            int64_t n = x + nb[0] * (y + nb[1] * z);
                            grow(&mn, &mx, raw[2 * n], raw[2 * n + 1]);
                        }
                int64_t c = cx + nc[0] * (cy + nc[1] * cz);
                craw[2 * c] = mn;
                craw[2 * c + 1] = mx;
            }
    /* ... combined with its +x/+y/+z coarse neighbours */
    for (int64_t cz = 0; cz < nc[2]; cz++)
        for (int64_t cy = 0; cy < nc[1]; cy++)
            for (int64_t cx = 0; cx < nc[0]; cx++) {
                float mn = INFINITY, mx = -INFINITY;
                for (int o = 0; o < 8; o++) {
                    int64_t x = cx + (o & 1), y = cy + ((o >> 1) & 1), z = cz + (o >> 2);
                    if (x >= nc[0] || y >= nc[1] || z >= nc[2]) continue;
                    int64_t n = x + nc[0] * (y + nc[1] * z);
                    grow(&mn, &mx, craw[2 * n], craw[2 * n + 1]);
                }
                int64_t c = cx + nc[0] * (cy + nc[1] * cz);
                coarse[2 * c] = mn;
                coarse[2 * c + 1] = mx;
            }

    if (!raw_out) free(raw);
    free(craw);
    return 0;
}
