/*
 * orc_sim.c -- progressive pass simulator with speculation and the LRU cache.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Replays the pass structure of Fig. 2 / Sec. 3 with the speculation of
 * Sec. 4 on the per-ray visible-block lists computed by orc_render:
 *   (a) every live ray takes its next k visible blocks (Sec. 3.3, 4.1);
 *   (b) the taken blocks are visible, they and their +x/+y/+z face, edge and
 *       corner neighbours are active (Sec. 3.4);
 *   (c) the active blocks go through the LRU cache: cached ones are touched,
 *       the others are decompressed into the least recently used slots not
 *       needed by this pass (Sec. 3.5);
 *   (e) a ray whose hit block is among its taken blocks finishes with a hit;
 *       a ray that got fewer than k blocks has left the volume and finishes
 *       without one (Sec. 4.4);
 *   (f) the remaining rays form the next pass's live list, in the order of
 *       the first live list.
 * k is the fixed count, or floor(w*h / N_Act) capped at k_max (Sec. 4), or,
 * for the per-ray count of Sec. 6's future work, ray p's own count in pass P
 * taken from a given table, capped by the pass's k_max (halved on overflow
 * like k); a ray that gets fewer blocks than its own count has left the
 * volume.
 *
 * Choices where the paper is silent (the cache of Sec. 3.5 grows instead):
 *   - LRU victims are the slots not used in this pass, ordered by the pass
 *     that used them last, then by slot index; misses are served in
 *     ascending block id.
 *   - When a pass needs more active blocks than the cache has slots, k is
 *     halved and the pass redone; at k = 1 the live list is cut to its first
 *     half instead, until the pass fits.  Neither changes the image.
 *   - The first live list holds the rays that enter the volume in screen
 *     tiles of 8 x 4 pixels, tiles left to right then top to bottom, pixels
 *     row by row inside a tile.  The order only decides which rays a cut
 *     live list keeps.
 */
#include "orc.h"

#include <stdlib.h>
#include <string.h>

int orc_spec_count(int64_t slots, int64_t n_active, int k_max)
{
    if (n_active <= 0) return 1;
    int64_t k = slots / n_active;
    if (k > k_max) k = k_max;
    if (k < 1) k = 1;
    return (int)k;
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

typedef struct { int64_t last; int64_t slot; } lru_key;

static int cmp_lru(const void *a, const void *b)
{
    const lru_key *x = (const lru_key *)a, *y = (const lru_key *)b;
    if (x->last != y->last) return (x->last > y->last) - (x->last < y->last);
    return (x->slot > y->slot) - (x->slot < y->slot);
}

/* ray p's count this attempt: the pass's k, or its own count (at least 1)
 * capped by it */
static int64_t ray_count(const int32_t *kp, int64_t p, int64_t kk)
{
    if (!kp) return kk;
    int64_t c = kp[p] < 1 ? 1 : kp[p];
    return c < kk ? c : kk;
}

/* sort and drop duplicates */
static int64_t uniq(uint32_t *v, int64_t n)
{
    if (n == 0) return 0;
    qsort(v, (size_t)n, sizeof *v, cmp_u32);
    int64_t m = 1;
    for (int64_t i = 1; i < n; i++)
        if (v[i] != v[m - 1]) v[m++] = v[i];
    return m;
}

int orc_simulate(int W, int H, const int32_t dims[3], const int32_t *enters,
                 const int32_t *hit_index, const int64_t *vis_off, const int32_t *n_vis,
                 const uint32_t *vis, int spec_mode, int k_fixed, int k_max, int64_t n_slots,
                 int max_passes, const int32_t *kray, orc_pass_stats *stats, int32_t *final_pass)
{
    int64_t npix = (int64_t)W * H;
    if (n_slots < 8 || k_fixed < 1 || k_max < 1) return -1;
    if (spec_mode == ORC_SPEC_PER_RAY && !kray) return -1;
    int64_t nb[3] = { (dims[0] + 3) / 4, (dims[1] + 3) / 4, (dims[2] + 3) / 4 };
    int64_t nblocks = nb[0] * nb[1] * nb[2];
    /* a cache with at least one slot per block never evicts; more slots than
     * blocks change nothing that is counted */
    if (n_slots > nblocks && nblocks >= 8) n_slots = nblocks;

    int64_t *live = malloc(sizeof(int64_t) * (npix + 1));
    int64_t *next = malloc(sizeof(int64_t) * (npix + 1));
    int64_t *pos = calloc((size_t)npix + 1, sizeof(int64_t));
    int64_t *blk_slot = malloc(sizeof(int64_t) * nblocks);
    int64_t *slot_blk = malloc(sizeof(int64_t) * n_slots);
    int64_t *slot_last = calloc((size_t)n_slots, sizeof(int64_t));
    lru_key *cand = malloc(sizeof(lru_key) * n_slots);
    if (!live || !next || !pos || !blk_slot || !slot_blk || !slot_last || !cand) return -2;
    for (int64_t b = 0; b < nblocks; b++) blk_slot[b] = -1;
    for (int64_t s = 0; s < n_slots; s++) slot_blk[s] = -1;
    if (final_pass) memset(final_pass, 0, sizeof(int32_t) * npix);

    int64_t n_live = 0;
    for (int ty = 0; ty < H; ty += 4)
        for (int tx = 0; tx < W; tx += 8)
            for (int y = ty; y < ty + 4 && y < H; y++)
                for (int x = tx; x < tx + 8 && x < W; x++) {
                    int64_t p = (int64_t)y * W + x;
                    if (enters[p]) live[n_live++] = p;
                }

    int pass = 0, rc = 0;
    uint32_t *vis_set = NULL, *act_set = NULL;
    while (n_live > 0 && pass < max_passes) {
        pass++;
        orc_pass_stats st;
        memset(&st, 0, sizeof st);
        st.pass = pass;
        st.n_active = n_live;
        int k = spec_mode == ORC_SPEC_FIXED      ? k_fixed
                : spec_mode == ORC_SPEC_PER_RAY ? k_max
                                                : orc_spec_count(npix, n_live, k_max);
        const int32_t *kp = spec_mode == ORC_SPEC_PER_RAY ? kray + (int64_t)(pass - 1) * npix : NULL;
        st.k = k;
        int kk = k;
        int64_t nproc = n_live, nvis = 0, nact = 0;

        for (;;) {
            /* (a)+(b): entries, visible and active sets */
            int64_t cap = 0;
            for (int64_t i = 0; i < nproc; i++) {
                int64_t p = live[i], avail = n_vis[p] - pos[p], kr = ray_count(kp, p, kk);
                cap += avail < kr ? avail : kr;
            }
            free(vis_set);
            free(act_set);
            vis_set = malloc(sizeof(uint32_t) * (cap + 1));
            act_set = malloc(sizeof(uint32_t) * (8 * cap + 1));
            nvis = 0;
            for (int64_t i = 0; i < nproc; i++) {
                int64_t p = live[i], avail = n_vis[p] - pos[p], kr = ray_count(kp, p, kk);
                int64_t take = avail < kr ? avail : kr;
                for (int64_t j = 0; j < take; j++) vis_set[nvis++] = vis[vis_off[p] + pos[p] + j];
            }
            st.n_entries = nvis;
            nvis = uniq(vis_set, nvis);
            nact = 0;
            for (int64_t i = 0; i < nvis; i++) {
                int64_t b = vis_set[i];
                int64_t bx = b % nb[0], by = (b / nb[0]) % nb[1], bz = b / (nb[0] * nb[1]);
                for (int o = 0; o < 8; o++) {
                    int64_t x = bx + (o & 1), y = by + ((o >> 1) & 1), z = bz + (o >> 2);
                    if (x >= nb[0] || y >= nb[1] || z >= nb[2]) continue;
                    act_set[nact++] = (uint32_t)(x + nb[0] * (y + nb[1] * z));
                }
            }
            nact = uniq(act_set, nact);
            if (nact <= n_slots) break;
            st.retries++;
            if (kk > 1) kk /= 2;
            else nproc = nproc > 1 ? nproc / 2 : 1;
        }
        st.k_used = kk;
        st.n_processed = nproc;
        st.n_visible = nvis;
        st.n_requested = nact;

        /* (c) the LRU cache: touch hits, then serve misses in block order */
        int64_t nmiss = 0;
        for (int64_t i = 0; i < nact; i++) {
            int64_t s = blk_slot[act_set[i]];
            if (s >= 0) slot_last[s] = pass;
            else act_set[nmiss++] = act_set[i]; /* misses, still ascending */
        }
        int64_t ncand = 0;
        for (int64_t s = 0; s < n_slots && nmiss > 0; s++)
            if (slot_last[s] < pass) {
                cand[ncand].last = slot_last[s];
                cand[ncand].slot = s;
                ncand++;
            }
        qsort(cand, (size_t)ncand, sizeof *cand, cmp_lru);
        if (ncand < nmiss) {
            rc = -3; /* cannot happen: nact <= n_slots */
            break;
        }
        for (int64_t i = 0; i < nmiss; i++) {
            int64_t s = cand[i].slot;
            if (slot_blk[s] >= 0) {
                blk_slot[slot_blk[s]] = -1;
                st.n_evicted++;
            }
            slot_blk[s] = act_set[i];
            blk_slot[act_set[i]] = s;
            slot_last[s] = pass;
        }
        st.n_decoded = nmiss;

        /* (e)+(f): terminate, compact the live list in order */
        int64_t n_next = 0;
        for (int64_t i = 0; i < n_live; i++) {
            int64_t p = live[i];
            if (i >= nproc) {
                next[n_next++] = p;
                continue;
            }
            int64_t avail = n_vis[p] - pos[p], kr = ray_count(kp, p, kk);
            int64_t take = avail < kr ? avail : kr;
            if (hit_index[p] >= 0 && hit_index[p] < pos[p] + take) {
                st.n_term_hit++;
                if (final_pass) final_pass[p] = pass;
            } else if (take < kr) {
                st.n_term_miss++;
                if (final_pass) final_pass[p] = pass;
            } else {
                pos[p] += take;
                next[n_next++] = p;
            }
        }
        int64_t *tmp = live;
        live = next;
        next = tmp;
        n_live = n_next;
        if (stats) stats[pass - 1] = st;
    }
    free(vis_set);
    free(act_set);
    free(live);
    free(next);
    free(pos);
    free(blk_slot);
    free(slot_blk);
    free(slot_last);
    free(cand);
    return rc ? rc : pass;
}

/* struct sizes, so that bindings can check their layouts */
int orc_sizeof_pixel(void) { return (int)sizeof(orc_pixel); }
int orc_sizeof_pass_stats(void) { return (int)sizeof(orc_pass_stats); }
int orc_sizeof_volume(void) { return (int)sizeof(orc_volume); }
