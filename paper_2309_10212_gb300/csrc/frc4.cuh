// frc4.cuh -- device encoder/decoder of the FRC4 fixed-rate 4^3 block codec.
//
// FRC4 is the project's stand-in for the ZFP fixed-rate mode the paper
// decompresses block by block on the GPU (Sec. 3.1, 3.5); the format is
// specified in spr.h.  Decoding runs one thread per block: the bit-plane
// parse scatters set bits into a private shared-memory column (one 32-bit
// word per coefficient, stride-padded so a warp's 32 columns hit 32 banks),
// then the 64 coefficients are pulled into registers for the inverse lifting
// transform, so every register index is static.
#pragma once

#include <stdint.h>

namespace spr {
namespace frc4 {

constexpr int kPlanes = 30;

// sequency order: (level(x)+level(y)+level(z), z, y, x), level = 0,1,2,2
struct Order {
    uint8_t v[64];
};
__host__ __device__ constexpr int level_of(int p) { return p == 0 ? 0 : (p == 1 ? 1 : 2); }
__host__ __device__ constexpr Order make_order()
{
    Order o{};
    int k = 0;
    for (int s = 0; s <= 6; ++s)
        for (int i = 0; i < 64; ++i) {
            // i = x + 4y + 16z enumerates z, then y, then x in ascending order
            int x = i & 3, y = (i >> 2) & 3, z = i >> 4;
            if (level_of(x) + level_of(y) + level_of(z) == s) o.v[k++] = (uint8_t)i;
        }
    return o;
}

// Bit sources: bits [pos, pos+n) of a block's little-endian stream, n <= 32.
// Reads past the end of the stream return zeros.
struct MemBits {   // any rate: 32-bit words read through the read-only path
    const uint32_t *w;
    int nwords;
    __device__ __forceinline__ uint32_t operator()(int pos, int n) const
    {
        int wi = pos >> 5;
        uint32_t lo = __ldg(w + wi);
        uint32_t hi = (wi + 1 < nwords) ? __ldg(w + wi + 1) : 0u;
        uint32_t v = __funnelshift_r(lo, hi, pos & 31);
        return n >= 32 ? v : (v & ((1u << n) - 1u));
    }
};

struct RegBits {   // rate <= 2: the whole 64- or 128-bit stream in registers, w0 first
    uint32_t w0, w1, w2, w3;
    // words pos/32 and pos/32 + 1 (pos < 128) picked by two selects per bit
    // of the word index, then one funnel shift
    __device__ __forceinline__ uint32_t operator()(int pos, int n) const
    {
        const bool k2 = (pos & 64) != 0, k1 = (pos & 32) != 0;
        const uint32_t x0 = k2 ? w2 : w0, x1 = k2 ? w3 : w1, x2 = k2 ? 0u : w2;
        const uint32_t v = __funnelshift_r(k1 ? x1 : x0, k1 ? x2 : x1, (uint32_t)pos);
        return n >= 32 ? v : (v & ((1u << n) - 1u));
    }
};

__device__ __forceinline__ RegBits load_reg_bits(const uint8_t *blk, int rate)
{
    RegBits b;
    if (rate == 2) {
        uint4 q = __ldg(reinterpret_cast<const uint4 *>(blk));
        b = RegBits{q.x, q.y, q.z, q.w};
    } else {
        uint2 q = __ldg(reinterpret_cast<const uint2 *>(blk));
        b = RegBits{q.x, q.y, 0u, 0u};
    }
    return b;
}

// Set bit p of a coefficient word in shared memory.  In a row (stride 1,
// decode_list_kernel) with an atomic OR: the thread issues it and moves on,
// where a load-or-store sequence would wait for the load of every set bit
// (no other thread touches the word).  In the strided columns of the range
// pass the atomics measured 5.6x slower than the load-or-store.
__device__ __forceinline__ void set_bit_of(uint32_t *w, int p, int stride)
{
    if (stride == 1) atomicOr(w, 1u << p);
    else *w |= 1u << p;
}

// Parse one block.  col[k * stride] receives the negabinary value of the k-th
// coefficient in sequency order (stride 1: col is 16-byte aligned).  Returns
// false for an all-zero block.  With nplanes given, *nplanes receives the
// number of bit planes parsed (0 for an all-zero block): the parse's length,
// by which the renderer's decoder groups blocks so that a warp's lanes run
// the plane loop alike.
template <class Bits>
__device__ __forceinline__ bool decode_coeffs(const Bits &bits_at, int rate, uint32_t *col, int stride,
                                              int *emax, int *nplanes = nullptr)
{
    if (stride == 1) {   // a row (16-byte aligned): vector stores
#pragma unroll
        for (int q = 0; q < 16; ++q) reinterpret_cast<uint4 *>(col)[q] = make_uint4(0u, 0u, 0u, 0u);
    } else {
#pragma unroll
        for (int i = 0; i < 64; ++i) col[i * stride] = 0u;
    }
    uint32_t h = bits_at(0, 9);
    if (!(h & 1u)) {
        if (nplanes) *nplanes = 0;
        return false;
    }
    int e = (int)((h >> 1) & 0xFFu) - 127;
    *emax = e < -100 ? -100 : e;
    int pos = 9, budget = 64 * rate - 9, n = 0;
    int p = kPlanes - 1;
    for (; p >= 0 && budget > 0; --p) {
        // refinement bits of the significant prefix
        int m = n < budget ? n : budget;
        for (int base = 0; base < m; base += 32) {
            int cnt = m - base < 32 ? m - base : 32;
            uint32_t bits = bits_at(pos + base, cnt);
            while (bits) {
                int i = __ffs(bits) - 1;
                bits &= bits - 1;
                set_bit_of(col + (base + i) * stride, p, stride);
            }
        }
        pos += m;
        budget -= m;
        // group tests and significance runs: one 32-bit read gives the test
        // bit (bit 0) and the first 31 bits of the run after it
        while (n < 64 && budget > 0) {
            const uint32_t w = bits_at(pos, 32);
            ++pos;
            --budget;
            if (!(w & 1u)) break;
            const int lim = 64 - n < budget ? 64 - n : budget;
            uint32_t run = w >> 1;
            if (lim < 31) run &= (1u << lim) - 1u;
            int used;
            bool found = run != 0u;
            if (found) {
                used = __ffs(run);
            } else {
                used = lim < 31 ? lim : 31;
                while (used < lim) {   // a run longer than the window
                    int cnt = lim - used < 32 ? lim - used : 32;
                    uint32_t bits = bits_at(pos + used, cnt);
                    if (bits) {
                        used += __ffs(bits);
                        found = true;
                        break;
                    }
                    used += cnt;
                }
            }
            pos += used;
            budget -= used;
            n += used;
            if (found) set_bit_of(col + (n - 1) * stride, p, stride);
        }
    }
    if (nplanes) *nplanes = kPlanes - 1 - p;
    return true;
}

// decode block `blk` (8*rate bytes, 16-byte aligned when rate == 2)
__device__ __forceinline__ bool decode_block_coeffs(const uint8_t *blk, int rate, uint32_t *col, int stride,
                                                    int *emax, int *nplanes = nullptr)
{
    if (rate <= 2) return decode_coeffs(load_reg_bits(blk, rate), rate, col, stride, emax, nplanes);
    return decode_coeffs(MemBits{reinterpret_cast<const uint32_t *>(blk), 2 * rate}, rate, col, stride, emax,
                         nplanes);
}

// two-level inverse lifting on one 4-vector, wrap-around integer arithmetic
__device__ __forceinline__ void inv_lift(int32_t &a0, int32_t &a1, int32_t &a2, int32_t &a3)
{
    int32_t ss = a0, dd = a1, d0 = a2, d1 = a3;
    int32_t s0 = (int32_t)((uint32_t)ss - (uint32_t)(dd >> 1));
    int32_t s1 = (int32_t)((uint32_t)s0 + (uint32_t)dd);
    a0 = (int32_t)((uint32_t)s0 - (uint32_t)(d0 >> 1));
    a1 = (int32_t)((uint32_t)a0 + (uint32_t)d0);
    a2 = (int32_t)((uint32_t)s1 - (uint32_t)(d1 >> 1));
    a3 = (int32_t)((uint32_t)a2 + (uint32_t)d1);
}

__device__ __forceinline__ void fwd_lift(int32_t &a0, int32_t &a1, int32_t &a2, int32_t &a3)
{
    int32_t d0 = (int32_t)((uint32_t)a1 - (uint32_t)a0);
    int32_t s0 = (int32_t)((uint32_t)a0 + (uint32_t)(d0 >> 1));
    int32_t d1 = (int32_t)((uint32_t)a3 - (uint32_t)a2);
    int32_t s1 = (int32_t)((uint32_t)a2 + (uint32_t)(d1 >> 1));
    int32_t dd = (int32_t)((uint32_t)s1 - (uint32_t)s0);
    int32_t ss = (int32_t)((uint32_t)s0 + (uint32_t)(dd >> 1));
    a0 = ss;
    a1 = dd;
    a2 = d0;
    a3 = d1;
}

__device__ __forceinline__ int32_t from_negabinary(uint32_t u)
{
    return (int32_t)((u ^ 0xAAAAAAAAu) - 0xAAAAAAAAu);
}

__device__ __forceinline__ uint32_t to_negabinary(int32_t x)
{
    return ((uint32_t)x + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}

// exact power of two as float, e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Coefficients in col (sequency order, negabinary) -> 64 floats in v.  The
// order table is a compile-time constant, so c[] is indexed statically.
__device__ __forceinline__ void reconstruct(const uint32_t *col, int stride, int emax, float v[64])
{
    constexpr Order ord = make_order();
    int32_t c[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) c[ord.v[k]] = from_negabinary(col[k * stride]);
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) inv_lift(c[x + 4 * y], c[x + 4 * y + 16], c[x + 4 * y + 32], c[x + 4 * y + 48]);
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) inv_lift(c[x + 16 * z], c[x + 16 * z + 4], c[x + 16 * z + 8], c[x + 16 * z + 12]);
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) inv_lift(c[4 * y + 16 * z], c[4 * y + 16 * z + 1], c[4 * y + 16 * z + 2], c[4 * y + 16 * z + 3]);
    float scale = pow2f(emax - 24);
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __fmul_rn(__int2float_rn(c[i]), scale);
}

// reconstruct() for coefficients in row[0..63] (16-byte aligned), read with
// 128-bit loads
__device__ __forceinline__ void reconstruct_row(const uint32_t *row, int emax, float v[64])
{
    constexpr Order ord = make_order();
    uint32_t u[64];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint4 w = reinterpret_cast<const uint4 *>(row)[q];
        u[4 * q] = w.x;
        u[4 * q + 1] = w.y;
        u[4 * q + 2] = w.z;
        u[4 * q + 3] = w.w;
    }
    int32_t c[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) c[ord.v[k]] = from_negabinary(u[k]);
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) inv_lift(c[x + 4 * y], c[x + 4 * y + 16], c[x + 4 * y + 32], c[x + 4 * y + 48]);
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) inv_lift(c[x + 16 * z], c[x + 16 * z + 4], c[x + 16 * z + 8], c[x + 16 * z + 12]);
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) inv_lift(c[4 * y + 16 * z], c[4 * y + 16 * z + 1], c[4 * y + 16 * z + 2], c[4 * y + 16 * z + 3]);
    float scale = pow2f(emax - 24);
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __fmul_rn(__int2float_rn(c[i]), scale);
}

// ------------------------------------------------------------------ encoder
struct BitWriter {
    uint32_t *out;
    int nwords;
    int widx;
    uint64_t acc;
    int nacc;
    __device__ void put(uint64_t bits, int n)  // n <= 32
    {
        acc |= (bits & ((n >= 64) ? ~0ull : ((1ull << n) - 1ull))) << nacc;
        nacc += n;
        while (nacc >= 32) {
            if (widx < nwords) out[widx] = (uint32_t)acc;
            ++widx;
            acc >>= 32;
            nacc -= 32;
        }
    }
    __device__ void put64(uint64_t bits, int n)  // n <= 64
    {
        if (n > 32) {
            put(bits & 0xFFFFFFFFull, 32);
            put(bits >> 32, n - 32);
        } else {
            put(bits, n);
        }
    }
    __device__ void finish()
    {
        if (nacc > 0) {
            if (widx < nwords) out[widx] = (uint32_t)acc;
            ++widx;
        }
        for (; widx < nwords; ++widx) out[widx] = 0u;
    }
};

// Encode 64 values (block positions) into 2*rate words.  Returns false for a
// non-finite input (the block is then written as zeros).
__device__ __forceinline__ bool encode_block(const float v[64], int rate, uint32_t *out)
{
    BitWriter bw{out, 2 * rate, 0, 0ull, 0};
    int emax = -1000;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        finite &= isfinite(v[i]);
        if (v[i] != 0.0f) {
            int e;
            frexpf(v[i], &e);
            emax = e > emax ? e : emax;
        }
    }
    if (!finite || emax == -1000) {
        bw.put(0, 1);
        bw.finish();
        return finite;
    }
    if (emax < -100) emax = -100;
    bw.put(1, 1);
    bw.put((uint32_t)(emax + 127), 8);
    float scale = pow2f(24 - emax);
    int32_t c[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) c[i] = __float2int_rn(__fmul_rn(v[i], scale));
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) fwd_lift(c[4 * y + 16 * z], c[4 * y + 16 * z + 1], c[4 * y + 16 * z + 2], c[4 * y + 16 * z + 3]);
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) fwd_lift(c[x + 16 * z], c[x + 16 * z + 4], c[x + 16 * z + 8], c[x + 16 * z + 12]);
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) fwd_lift(c[x + 4 * y], c[x + 4 * y + 16], c[x + 4 * y + 32], c[x + 4 * y + 48]);
    constexpr Order ord = make_order();
    uint32_t u[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) u[k] = to_negabinary(c[ord.v[k]]);

    int budget = 64 * rate - 9, n = 0;
    for (int p = kPlanes - 1; p >= 0 && budget > 0; --p) {
        uint64_t x = 0;
#pragma unroll
        for (int k = 0; k < 64; ++k) x |= (uint64_t)((u[k] >> p) & 1u) << k;
        int m = n < budget ? n : budget;
        bw.put64(x, m);
        budget -= m;
        while (n < 64 && budget > 0) {
            uint64_t rest = x >> n;
            bw.put(rest != 0, 1);
            --budget;
            if (!rest) break;
            int lim = 64 - n < budget ? 64 - n : budget;
            int z = __ffsll((long long)rest) - 1;
            if (z + 1 <= lim) {
                bw.put64(1ull << z, z + 1);
                n += z + 1;
                budget -= z + 1;
            } else {
                bw.put64(0, lim);
                n += lim;
                budget -= lim;
            }
        }
    }
    bw.finish();
    return true;
}

}  // namespace frc4
}  // namespace spr
