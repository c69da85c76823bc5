// packed.cu -- zero-suppressed table levels (the count tables of Section
// 3.2.1: per node only the non-zero entries, sorted by key) with optional
// variable-length counts (Section 3.3.3: each row stores its counts in the
// fewest of 1, 2, 4, 8 or 16 bytes that hold its largest count).  Built from
// the dense levels once the table build is done; the sampler then reads
// entries by binary search of a row's keys (packed_get).
#include "internal.h"

namespace mc {

void inclusive_scan_u128(u128 *x, int64_t n, int *err, Arena &scratch, cudaStream_t s);

__device__ __forceinline__ int count_bytes(u128 x)
{
    if ((x >> 64) != 0) return 16;
    const uint64_t y = (uint64_t)x;
    if (y >> 32) return 8;
    if (y >> 16) return 4;
    if (y >> 8) return 2;
    return 1;
}

__device__ __forceinline__ void store_count(uint8_t *q, u128 x, int w)
{
    switch (w) {
    case 1: q[0] = (uint8_t)x; break;
    case 2: *(uint16_t *)q = (uint16_t)x; break;
    case 4: *(uint32_t *)q = (uint32_t)x; break;
    case 8: *(uint64_t *)q = (uint64_t)x; break;
    default:
        ((uint64_t *)q)[0] = (uint64_t)x;
        ((uint64_t *)q)[1] = (uint64_t)(x >> 64);
    }
}

__device__ __forceinline__ u128 warp_max(u128 x)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const u128 y = shfl_xor(x, d);
        if (y > x) x = y;
    }
    return x;
}

// Pass 1, a warp per node: the row's non-zero entries, the bytes per count
// (varlen: the row's own width, else the table's) and the row's count bytes
// rounded up to 8.
template <typename CT>
__global__ void pack_count_kernel(const CT *__restrict__ D, int64_t n, int W, int varlen, u128 *cnt,
                                  u128 *bytes, uint8_t *wid)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < n; v += nw) {
        unsigned nz = 0;
        u128 mx = 0;
        for (int e = lane; e < W; e += 32) {
            const u128 x = widen(D[v * W + e]);
            nz += x != 0;
            if (x > mx) mx = x;
        }
        for (int d = 16; d > 0; d >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, d);
        mx = warp_max(mx);
        if (lane == 0) {
            const int w = varlen ? count_bytes(mx) : (int)sizeof(CT);
            cnt[v] = nz;
            bytes[v] = ((u128)nz * w + 7) & ~(u128)7;
            if (wid) wid[v] = (uint8_t)w;
        }
    }
}

// Exclusive int64 offsets (n + 1 of them) from an inclusive u128 prefix.
__global__ void offsets_kernel(const u128 *__restrict__ inc, int64_t n, int64_t *__restrict__ off)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x)
        off[v] = v == 0 ? 0 : (int64_t)inc[v - 1];
}

// Pass 2, a warp per node: keys and counts of the non-zero entries, in row
// order.
template <typename CT>
__global__ void pack_fill_kernel(const CT *__restrict__ D, int64_t n, int W, PackedView p, uint16_t *__restrict__ key,
                                 uint8_t *__restrict__ val)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < n; v += nw) {
        const int64_t o0 = p.off[v];
        const int w = p.wid ? (int)p.wid[v] : p.width;
        uint8_t *q0 = val + p.boff[v];
        int64_t base = 0;
        for (int e0 = 0; e0 < W; e0 += 32) {
            const int e = e0 + lane;
            const u128 x = e < W ? widen(D[v * W + e]) : (u128)0;
            const unsigned m = __ballot_sync(0xffffffffu, x != 0);
            if (x != 0) {
                const int64_t j = base + __popc(m & lt);
                key[o0 + j] = (uint16_t)e;
                store_count(q0 + j * w, x, w);
            }
            base += __popc(m);
        }
    }
}

// Per-node totals over the allowed shapes (entry e of a set-major row is
// shape e % R), a warp per node.
__global__ void packed_row_totals_kernel(PackedView p, int64_t n, int R, uint64_t allow0, uint64_t allow1,
                                         u128 *__restrict__ tot, int *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool ovf = false;
    for (int64_t v = w0; v < n; v += nw) {
        const int64_t lo = p.off[v], hi = p.off[v + 1];
        const int w = p.wid ? (int)p.wid[v] : p.width;
        const uint8_t *q0 = p.val + p.boff[v];
        u128 s = 0;
        for (int64_t j = lo + lane; j < hi; j += 32) {
            const int sh = (int)p.key[j] % R;
            const bool ok = sh < 64 ? (allow0 >> sh) & 1 : (allow1 >> (sh - 64)) & 1;
            if (ok) ovf |= add_ovf(s, packed_value(q0 + (j - lo) * w, w));
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ovf |= add_ovf(s, shfl_xor(s, d));
        if (lane == 0) tot[v] = s;
    }
    if (ovf) atomicOr(err, 1);
}

// Dense rows from packed ones, a warp per node.
template <typename CT>
__global__ void unpack_kernel(PackedView p, int64_t n, int W, CT *__restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < n; v += nw) {
        for (int e = lane; e < W; e += 32) dst[v * W + e] = 0;
        __syncwarp();
        const int64_t lo = p.off[v], hi = p.off[v + 1];
        const int w = p.wid ? (int)p.wid[v] : p.width;
        const uint8_t *q0 = p.val + p.boff[v];
        for (int64_t j = lo + lane; j < hi; j += 32) dst[v * W + p.key[j]] = (CT)packed_value(q0 + (j - lo) * w, w);
    }
}

template <typename CT>
static PackedView pack_level(mc_tables *t, const void *dense, int W, cudaStream_t s, int64_t &stored)
{
    const int64_t n = t->g->n;
    Arena scratch(true);
    scratch.alloc = t->arena.alloc;
    scratch.stream = s;
    int *err = scratch.get<int>(1);
    MC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    u128 *cnt = scratch.get<u128>((size_t)n);
    u128 *bytes = scratch.get<u128>((size_t)n);
    PackedView p;
    p.width = (int)sizeof(CT);
    uint8_t *wid = t->varlen ? t->arena.get<uint8_t>((size_t)n) : nullptr;
    const int grid = grid_for(n * 32, 256);
    MC_LAUNCH("pack", s, pack_count_kernel<CT><<<grid, 256, 0, s>>>((const CT *)dense, n, W, t->varlen ? 1 : 0, cnt,
                                                                      bytes, wid));
    inclusive_scan_u128(cnt, n, err, scratch, s);
    inclusive_scan_u128(bytes, n, err, scratch, s);
    int64_t *off = t->arena.get<int64_t>((size_t)n + 1);
    int64_t *boff = t->arena.get<int64_t>((size_t)n + 1);
    MC_LAUNCH("pack", s, offsets_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(cnt, n, off));
    MC_LAUNCH("pack", s, offsets_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(bytes, n, boff));
    int64_t tail[2] = {0, 0};
    int herr = 0;
    MC_CUDA(cudaMemcpyAsync(&tail[0], off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(&tail[1], boff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error(MC_E_INTERNAL, "packing: offset overflow");
    uint16_t *key = t->arena.get<uint16_t>((size_t)std::max<int64_t>(tail[0], 1));
    uint8_t *val = t->arena.get<uint8_t>((size_t)std::max<int64_t>(tail[1], 8));
    p.off = off;
    p.boff = boff;
    p.wid = wid;
    p.key = key;
    p.val = val;
    MC_LAUNCH("pack", s, pack_fill_kernel<CT><<<grid, 256, 0, s>>>((const CT *)dense, n, W, p, key, val));
    stored += tail[0] * 2 + tail[1] + 16 * (n + 1) + (wid ? n : 0);
    return p;
}

void pack_tables(mc_tables *t, cudaStream_t s)
{
    const int64_t n = t->g->n;
    const size_t cb = t->bits / 8;
    int64_t dense = 0, stored = 0;
    for (int which = 0; which < 2; ++which)
        for (int h = which ? 1 : 2; h <= (which ? t->k - 1 : t->k); ++h) {
            if (t->level_missing(h)) continue;
            void *&D = which ? t->S[h] : t->c[h];
            const int W = which ? t->geo.Ws[h] : t->geo.Wc[h];
            dense += n * W * (int64_t)cb;
            if (n == 0) continue;
            PackedView p = t->bits == 64 ? pack_level<uint64_t>(t, D, W, s, stored)
                                         : pack_level<u128>(t, D, W, s, stored);
            (which ? t->ps : t->pc)[h] = p;
            MC_CUDA(cudaStreamSynchronize(s));
            t->arena.release(D);
            D = nullptr;
        }
    t->dense_bytes = dense;
    t->stored_bytes = stored;
}

void launch_packed_row_totals(const mc_tables *t, int h, uint64_t allow0, uint64_t allow1, u128 *tot, int *err,
                              cudaStream_t s)
{
    const int64_t n = t->g->n;
    if (n == 0) return;
    MC_LAUNCH("row_totals", s, packed_row_totals_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(
                                   t->pc[h], n, shape_catalog().r[h], allow0, allow1, tot, err));
}

void launch_unpack(const mc_tables *t, int h, int which, void *dst, cudaStream_t s)
{
    const int64_t n = t->g->n;
    if (n == 0) return;
    const PackedView &p = which ? t->ps[h] : t->pc[h];
    const int W = which ? t->geo.Ws[h] : t->geo.Wc[h];
    if (t->bits == 64)
        MC_LAUNCH("unpack", s, unpack_kernel<uint64_t><<<grid_for(n * 32, 256), 256, 0, s>>>(p, n, W, (uint64_t *)dst));
    else
        MC_LAUNCH("unpack", s, unpack_kernel<u128><<<grid_for(n * 32, 256), 256, 0, s>>>(p, n, W, (u128 *)dst));
}

}  // namespace mc

using namespace mc;

extern "C" mc_status mc_table_bytes(const mc_tables *t, int64_t *dense_bytes, int64_t *stored_bytes)
{
    return guarded([&] {
        MC_REQUIRE(t, "tables is NULL");
        int64_t dense = t->dense_bytes, stored = t->stored_bytes;
        if (!t->packed) {
            dense = 0;
            const int64_t n = t->g->n;
            for (int h = 2; h <= t->k; ++h)
                if (!t->level_missing(h)) dense += n * t->geo.Wc[h] * (int64_t)(t->bits / 8);
            for (int h = 1; h < t->k; ++h)
                if (!t->level_missing(h)) dense += n * t->geo.Ws[h] * (int64_t)(t->bits / 8);
            stored = dense;
        }
        if (dense_bytes) *dense_bytes = dense;
        if (stored_bytes) *stored_bytes = stored;
    });
}
