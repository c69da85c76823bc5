// common.cuh -- device helpers shared by the library's kernels: exact
// unsigned counts with overflow detection, Philox4x32-10, colour-set ranks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mc {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Exact counts.  A count type CT is uint64_t or u128; every add and multiply
// reports whether the true result fits.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ bool add_ovf(uint64_t &acc, uint64_t x)
{
    acc += x;
    return acc < x;
}
__host__ __device__ __forceinline__ bool add_ovf(u128 &acc, u128 x)
{
    acc += x;
    return acc < x;
}

__device__ __forceinline__ bool mul_ovf(uint64_t a, uint64_t b, uint64_t &p)
{
    p = a * b;
    return __umul64hi(a, b) != 0;
}

__device__ __forceinline__ bool mul_ovf(u128 a, u128 b, u128 &p)
{
    const uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64);
    const uint64_t b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    const uint64_t lo = a0 * b0, hi0 = __umul64hi(a0, b0);
    if (a1 == 0 && b1 == 0) {
        p = ((u128)hi0 << 64) | lo;
        return false;
    }
    if (a1 != 0 && b1 != 0) { p = 0; return true; }
    const uint64_t x = a1 ? a1 : b1, y = a1 ? b0 : a0;
    if (__umul64hi(x, y) != 0) { p = 0; return true; }
    const uint64_t cross = x * y;
    const uint64_t hi = hi0 + cross;
    p = ((u128)hi << 64) | lo;
    return hi < cross;
}

// Exact division by beta in {1..8}: x / beta = (x >> t) * inv(beta >> t)
// mod 2^w with t = ctz(beta); the quotient is checked to be exact (the
// divisibility test of Granlund and Montgomery: q * b' == x' and q <= max/b').
struct ExactDiv {
    u128 inv128, qmax128;   // inverse of the odd part mod 2^128; (2^128-1) / odd part
    uint64_t inv64, qmax64; // the same mod 2^64
    int shift;              // trailing zeros of beta
    int pad_[3];
};

__device__ __forceinline__ bool exact_div(uint64_t x, const ExactDiv &d, uint64_t &q)
{
    if (x & ((1ull << d.shift) - 1)) return false;
    q = (x >> d.shift) * d.inv64;
    return q <= d.qmax64;
}
__device__ __forceinline__ bool exact_div(u128 x, const ExactDiv &d, u128 &q)
{
    if ((uint64_t)x & ((1ull << d.shift) - 1)) return false;
    q = (x >> d.shift) * d.inv128;
    return q <= d.qmax128;
}

template <typename CT> struct CountBits;
template <> struct CountBits<uint64_t> { static constexpr int value = 64; };
template <> struct CountBits<u128> { static constexpr int value = 128; };

__device__ __forceinline__ u128 widen(uint64_t x) { return (u128)x; }
__device__ __forceinline__ u128 widen(u128 x) { return x; }

// Warp shuffles of 128-bit values.
__device__ __forceinline__ u128 shfl_up(u128 x, int d)
{
    uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)x, d);
    uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(x >> 64), d);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_xor(u128 x, int d)
{
    uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)x, d);
    uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(x >> 64), d);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ uint64_t shfl_xor(uint64_t x, int d)
{
    return __shfl_xor_sync(0xffffffffu, x, d);
}
__device__ __forceinline__ uint64_t shfl_up(uint64_t x, int d)
{
    return __shfl_up_sync(0xffffffffu, x, d);
}
__device__ __forceinline__ uint64_t shfl(uint64_t x, int src)
{
    return __shfl_sync(0xffffffffu, x, src);
}
__device__ __forceinline__ u128 shfl(u128 x, int src)
{
    uint64_t lo = __shfl_sync(0xffffffffu, (uint64_t)x, src);
    uint64_t hi = __shfl_sync(0xffffffffu, (uint64_t)(x >> 64), src);
    return ((u128)hi << 64) | lo;
}

// Inclusive warp scan of 128-bit values (sums never exceed a checked bound).
__device__ __forceinline__ u128 warp_inclusive_scan(u128 x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u128 y = shfl_up(x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// u128 -> double, rounded to nearest even: the top 64 significant bits with
// the lower bits folded into a sticky bit, then one correctly rounded
// conversion and an exact scaling.
__device__ __forceinline__ double u128_to_double(u128 x)
{
    const uint64_t hi = (uint64_t)(x >> 64);
    if (hi == 0) return __ull2double_rn((uint64_t)x);
    const int nb = 128 - __clzll(hi);
    const int shift = nb - 64;
    uint64_t top = (uint64_t)(x >> shift);
    const u128 rest = x & ((((u128)1) << shift) - 1);
    if (rest != 0) top |= 1ull;
    return scalbn(__ull2double_rn(top), shift);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t x0 = (uint32_t)(m1 >> 32) ^ c[1] ^ k0;
        const uint32_t x2 = (uint32_t)(m0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)m1;
        c[3] = (uint32_t)m0;
        c[0] = x0;
        c[2] = x2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Uniform integer in [0, W), W >= 1: 128 Philox bits for counter
// (index_lo, index_hi, step, attempt), masked to the smallest power of two
// >= W, rejected and redrawn with attempt + 1 while >= W.  Each attempt is
// accepted with probability > 1/2; after 128 rejections (probability below
// 2^-128) or for W = 0 the draw reports failure instead of looping on.
__device__ __forceinline__ bool draw_below(uint64_t seed, uint64_t index, uint32_t step, u128 W, u128 &out)
{
    if (W == 0) return false;
    const u128 wm1 = W - 1;
    const uint64_t whi = (uint64_t)(wm1 >> 64), wlo = (uint64_t)wm1;
    const int bits = whi ? 128 - __clzll(whi) : 64 - __clzll(wlo);
    const u128 mask = bits >= 128 ? ~(u128)0 : ((((u128)1) << bits) - 1);
    for (uint32_t attempt = 0; attempt < 128; ++attempt) {
        uint32_t c[4] = {(uint32_t)index, (uint32_t)(index >> 32), step, attempt};
        philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        u128 r = (u128)c[0] | ((u128)c[1] << 32) | ((u128)c[2] << 64) | ((u128)c[3] << 96);
        r &= mask;
        if (r < W) { out = r; return true; }
    }
    return false;
}

// The same draw when W < 2^64: the mask keeps only the low 64 of the 128
// Philox bits, so the value is identical to the 128-bit draw above.
__device__ __forceinline__ bool draw_below(uint64_t seed, uint64_t index, uint32_t step, uint64_t W, uint64_t &out)
{
    if (W == 0) return false;
    const uint64_t wm1 = W - 1;
    const int bits = 64 - __clzll(wm1);
    const uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
    for (uint32_t attempt = 0; attempt < 128; ++attempt) {
        uint32_t c[4] = {(uint32_t)index, (uint32_t)(index >> 32), step, attempt};
        philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t r = ((uint64_t)c[0] | ((uint64_t)c[1] << 32)) & mask;
        if (r < W) { out = r; return true; }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Colour sets.  A set of colours is a bit mask (bit a = colour a).  Tables
// are colour-relative: at node v the colour c_v is deleted from the palette
// and higher colours move down by one; a set of the remaining k-1 colours is
// then indexed by its colex rank among sets of its size (colex order of sets
// is ascending order of their masks).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned drop_colour(unsigned mask, int c)
{
    return (mask & ((1u << c) - 1u)) | ((mask >> (c + 1)) << c);
}
__host__ __device__ __forceinline__ unsigned insert_colour_gap(unsigned rel, int c)
{
    return (rel & ((1u << c) - 1u)) | ((rel >> c) << (c + 1));
}

// ---------------------------------------------------------------------------
// Packed (zero-suppressed) table levels, Section 3.2.1: per node row only the
// non-zero entries, in row order, each as a key (the entry's index in the
// dense row) and a count.  Counts are stored at `width` bytes each when
// `wid` is NULL (the table's width), else at the row's own width wid[v]
// (1, 2, 4, 8 or 16 bytes: the fewest that hold the row's largest count, the
// variable-length counts of Section 3.3.3).  Row v's keys are
// key[off[v] .. off[v+1]), its counts start at byte boff[v] (a multiple of 8).
// ---------------------------------------------------------------------------
struct PackedView {
    const int64_t *off = nullptr;
    const int64_t *boff = nullptr;
    const uint8_t *wid = nullptr;
    const uint16_t *key = nullptr;
    const uint8_t *val = nullptr;
    int width = 8;
};

__device__ __forceinline__ u128 packed_value(const uint8_t *q, int w)
{
    switch (w) {
    case 1: return (u128)q[0];
    case 2: return (u128)*(const uint16_t *)q;
    case 4: return (u128)*(const uint32_t *)q;
    case 8: return (u128)*(const uint64_t *)q;
    default: return (u128)((const uint64_t *)q)[0] | ((u128)((const uint64_t *)q)[1] << 64);
    }
}

// Entry idx of row v (0 when it is not stored), by binary search of the
// row's keys.
__device__ __forceinline__ u128 packed_get(const PackedView &p, int64_t v, int idx)
{
    const int64_t lo = p.off[v], hi = p.off[v + 1];
    int64_t l = lo, r = hi;
    while (l < r) {
        const int64_t mid = (l + r) >> 1;
        if ((int)p.key[mid] < idx) l = mid + 1; else r = mid;
    }
    if (l >= hi || (int)p.key[l] != idx) return 0;
    const int w = p.wid ? (int)p.wid[v] : p.width;
    return packed_value(p.val + p.boff[v] + (l - lo) * w, w);
}

}  // namespace mc
