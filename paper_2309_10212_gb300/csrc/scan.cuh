// scan.cuh -- single-pass stream compaction / prefix sum with decoupled
// look-back (Merrill and Garland), the primitive behind the compactions and
// prefix sums of Sec. 3.6 and 4.2.  The look-back is warp-parallel: one warp
// inspects 32 predecessors per round.
//
// One kernel computes, for elements i in [0, n), a count c(i) and calls
// emit(i, prefix, c(i)) with the exclusive prefix sum of the counts.  Tiles
// take their index from an atomic ticket, so every tile a thread waits on is
// already running or done.  Each tile publishes its aggregate, then its
// inclusive prefix, in one 64-bit word: bits 63..62 = status (1 aggregate,
// 2 inclusive), bits 61..32 = the launch's epoch, bits 31..0 = value.  A
// word whose epoch is not the current one reads as "not yet published", so
// the status words need no clearing between launches: the last CTA to leave
// resets the ticket and advances the epoch (and clears every status word
// when the 30-bit epoch wraps).  Status words and the ticket/done/epoch
// words must be zero when first allocated.  Waits are bounded: after
// `spin_limit` polls (with nanosleep back-off) a tile sets the timeout flag
// and gives up, and every other waiting tile stops as soon as it sees it.
#pragma once

#include <stdint.h>

namespace spr {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int64_t kDefaultSpinLimit = int64_t(1) << 22;

struct ScanCtl {
    unsigned long long *status;  // one word per tile; zero when allocated
    int64_t n_status;            // words in status
    unsigned int *seq;           // [0] ticket, [1] CTAs done, [2] epoch; zero when allocated
    unsigned int *flags;         // bit 0: a wait timed out
    int64_t spin_limit;
    int64_t withhold;            // test hook: this tile never publishes (-1: none)
    uint32_t *over;              // optional: set to (total > over_limit) with the total
    uint32_t over_limit;
};

constexpr unsigned long long kAgg = 1ull << 62;
constexpr unsigned long long kInc = 2ull << 62;
constexpr unsigned long long kStatusBits = 3ull << 62;
constexpr unsigned long long kEpochBits = 0x3FFFFFFFull << 32;
constexpr unsigned int kEpochMask = 0x3FFFFFFFu;

__device__ __forceinline__ void publish(unsigned long long *w, unsigned long long v)
{
    atomicExch(w, v);
}

__device__ __forceinline__ unsigned long long poll(const unsigned long long *w)
{
    return *(const volatile unsigned long long *)w;
}

// n is read from *n_dev when n_dev is non-null (counts produced on the
// device), else n_host is used.  total (optional) receives the sum.
template <class CountF, class EmitF>
__global__ void __launch_bounds__(kScanThreads)
    compact_kernel(int64_t n_host, const uint32_t *n_dev, ScanCtl ctl, CountF count, EmitF emit,
                   uint32_t *total)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_prefix;
    __shared__ uint32_t s_total;
    __shared__ uint32_t s_epoch;
    __shared__ uint32_t s_last;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = threadIdx.x >> 5;
    if (!count.enabled()) return;
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    if (tid == 0) s_epoch = *(volatile unsigned int *)&ctl.seq[2] & kEpochMask;
    // persistent: each CTA takes tiles in ticket order until none is left, so
    // every tile a look-back waits on belongs to a running CTA
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctl.seq[0], 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        const int64_t base = tile * kScanTile;
        if (base >= n) {  // nobody waits on tiles past the end
            if (tile == 0 && tid == 0) {
                if (total) *total = 0u;
                if (ctl.over) *ctl.over = 0u;
            }
            break;
        }
        const unsigned long long tag = (unsigned long long)s_epoch << 32;

        uint32_t c[kScanItems];
        uint32_t local = 0;
        const int64_t first = base + (int64_t)tid * kScanItems;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t i = first + k;
            c[k] = i < n ? count(i) : 0u;
            local += c[k];
        }
        // block-wide exclusive scan of the per-thread sums
        uint32_t incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < kScanThreads / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
        }
        __syncthreads();
        uint32_t excl = s_warp[wid] + incl - local;
        if (tid == kScanThreads - 1) s_total = excl + local;
        __syncthreads();
        const uint32_t total_tile = s_total;

        // Look-back by warp 0: lane j inspects tile - 1 - j - 32r in round
        // r.  The nearest predecessor holding an inclusive prefix ends the
        // walk; every tile between it and this one must have published its
        // aggregate (else the warp waits and polls again).  One round covers
        // 32 predecessors, so tiles that run together do not wait on each
        // other's serial walks.
        if (wid == 0) {
            uint32_t prefix = 0;
            const bool publish_ok = tile != ctl.withhold;
            if (tile == 0) {
                if (lane == 0 && publish_ok) publish(&ctl.status[0], kInc | tag | total_tile);
            } else {
                if (lane == 0 && publish_ok) publish(&ctl.status[tile], kAgg | tag | total_tile);
                int64_t hi = tile - 1;   // nearest predecessor of this round's window
                int64_t polls = 0;
                unsigned ns = 32;
                bool gave_up = false;
                for (;;) {
                    const int64_t pred = hi - lane;
                    unsigned long long w = pred >= 0 ? poll(&ctl.status[pred]) : 0ull;
                    const unsigned long long st = w & kStatusBits;
                    const bool valid = pred >= 0 && st != 0 && (w & kEpochBits) == tag;
                    const unsigned inc = __ballot_sync(0xFFFFFFFFu, valid && st == kInc);
                    const unsigned ok = __ballot_sync(0xFFFFFFFFu, valid);
                    // lanes that must be valid: up to the nearest inclusive,
                    // or every lane with a predecessor when none is inclusive
                    const int first_inc = inc ? __ffs(inc) - 1 : 32;
                    const int span = hi + 1 < 32 ? (int)(hi + 1) : 32;
                    const int need_n = first_inc < 32 ? first_inc + 1 : span;
                    const unsigned need = need_n >= 32 ? 0xFFFFFFFFu : ((1u << need_n) - 1u);
                    if ((ok & need) != need) {
                        if (++polls > ctl.spin_limit) {
                            if (lane == 0) atomicOr(ctl.flags, 1u);
                            gave_up = true;
                        } else if ((polls & 63) == 0 && (*(volatile unsigned int *)ctl.flags & 1u)) {
                            gave_up = true;
                        }
                        if (__any_sync(0xFFFFFFFFu, gave_up)) break;
                        __nanosleep(ns);
                        if (ns < 256) ns <<= 1;
                        continue;
                    }
                    uint32_t v = (lane < need_n) ? (uint32_t)(w & 0xFFFFFFFFull) : 0u;
#pragma unroll
                    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                    prefix += v;
                    if (first_inc < 32 || hi < 32) break;
                    hi -= 32;
                }
                if (lane == 0 && publish_ok) publish(&ctl.status[tile], kInc | tag | (uint32_t)(prefix + total_tile));
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (base + kScanTile >= n) {
                    if (total) *total = prefix + total_tile;
                    if (ctl.over) *ctl.over = (prefix + total_tile) > ctl.over_limit ? 1u : 0u;
                }
            }
        }
        __syncthreads();
        uint32_t run = s_prefix + excl;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t i = first + k;
            if (i < n) emit(i, run, c[k]);
            run += c[k];
        }
        __syncthreads();   // shared state is reused by this CTA's next tile
    }
    // every CTA has taken its last ticket when the done count reaches the
    // grid size; that CTA resets the ticket and opens the next epoch
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl.seq[1], 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    const uint32_t next = (s_epoch + 1u) & kEpochMask;
    if (next == 0) {  // epoch wrap: no stale word may carry a reused epoch
        for (int64_t i = tid; i < ctl.n_status; i += kScanThreads) ctl.status[i] = 0ull;
        __threadfence();
        __syncthreads();
    }
    if (tid == 0) {
        atomicExch(&ctl.seq[0], 0u);
        atomicExch(&ctl.seq[1], 0u);
        __threadfence();
        atomicExch(&ctl.seq[2], next);
    }
}

inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

}  // namespace spr
