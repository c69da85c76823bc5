// gather.cuh -- the neighbour sums S_h(v) = sum over the neighbours u of v
// of c_h(u) (the inner sum over u of Eq. 1), the kernel shared by the
// translation units that instantiate it (gather_*.cu) and the table build.
#pragma once

#include "internal.h"

namespace mc {

enum : int { ERR_OVERFLOW = 1, ERR_INEXACT = 2, ERR_COLOUR = 4, ERR_SEARCH = 8 };

// ---------------------------------------------------------------------------
// Neighbour sums of level h >= 2 (the inner sum over u of Eq. 1):
//   S_h(v)[rho'', s] = sum_{u ~ v} c_h(u)[map(c_v, c_u, rho''), s].
// Rows are set-major, so the entries of one colour set (all r_h shapes) are
// contiguous, and a neighbour u contributes whole sets: the S sets holding
// c_u take u's sets that avoid c_v.  A row is handled in units of UB bytes
// (16 when a set's bytes are a multiple of 16, else 8); a lane owns S units
// j, j + G, ... of its node and, per neighbour, loads the one source unit
// that feeds each (map in shared memory), U neighbours in flight.
//   * nodes of degree <= HUB_CHUNK: G lanes per node, 32 / G nodes per warp,
//     taken in the order of `sched` (descending degree, so the nodes of a
//     warp have nearly equal degrees);
//   * hub chunks (HUB_CHUNK consecutive neighbours of a hub): a warp per
//     chunk, its 32 / G groups on different neighbours, summed by shuffles;
//     the partial row goes to `partial`, entry-major per hub.
// The first `chunk_blocks` blocks take the hub chunks, the rest the nodes.
// ---------------------------------------------------------------------------
struct GatherArgs {
    const int64_t *row_ptr;
    const uint32_t *col;
    const uint8_t *colors;
    const uint8_t *ecol;
    const uint4 *sched;      // nodes of degree <= HUB_CHUNK, descending degree: (v, e0 lo, e0 hi, degree)
    int64_t n_small;
    const int32_t *node_chunk0;
    const void *src;   // c_h, n x Wc
    void *dst;         // S_h, n x Ws
    void *partial;     // n_chunks x Ws
    const uint32_t *chunk_node;
    const int64_t *chunk_e0, *chunk_e1;
    const int16_t *gmap;
    int64_t n, n_chunks;
    int k, Bs, Wc, Ws;
    int ups;           // units per colour set
    int wc_units, ws_units;
    int chunk_blocks;
    int *err;
};

// A unit of UB bytes of a row of CT counts, with exact (overflow-checked) adds.
template <typename CT, int UB> struct Unit;
template <> struct Unit<uint64_t, 8> {
    uint64_t a;
    __device__ __forceinline__ void zero() { a = 0; }
    __device__ __forceinline__ void load(const void *p) { a = __ldg((const unsigned long long *)p); }
    __device__ __forceinline__ bool add(const Unit &x) { return add_ovf(a, x.a); }
    __device__ __forceinline__ void store(void *p) const { *(uint64_t *)p = a; }
    __device__ __forceinline__ Unit xor_shfl(int d) const { Unit r; r.a = __shfl_xor_sync(0xffffffffu, a, d); return r; }
    __device__ __forceinline__ uint64_t entry(int i) const { return a; }
};
template <> struct Unit<uint64_t, 16> {
    uint64_t a, b;
    __device__ __forceinline__ void zero() { a = b = 0; }
    __device__ __forceinline__ void load(const void *p)
    {
        const ulonglong2 v = __ldg((const ulonglong2 *)p);
        a = v.x;
        b = v.y;
    }
    __device__ __forceinline__ bool add(const Unit &x)
    {
        const bool o1 = add_ovf(a, x.a);
        const bool o2 = add_ovf(b, x.b);
        return o1 | o2;
    }
    __device__ __forceinline__ void store(void *p) const { *(ulonglong2 *)p = make_ulonglong2(a, b); }
    __device__ __forceinline__ Unit xor_shfl(int d) const
    {
        Unit r;
        r.a = __shfl_xor_sync(0xffffffffu, a, d);
        r.b = __shfl_xor_sync(0xffffffffu, b, d);
        return r;
    }
    __device__ __forceinline__ uint64_t entry(int i) const { return i ? b : a; }
};
template <> struct Unit<u128, 16> {
    u128 a;
    __device__ __forceinline__ void zero() { a = 0; }
    __device__ __forceinline__ void load(const void *p)
    {
        const ulonglong2 v = __ldg((const ulonglong2 *)p);
        a = ((u128)v.y << 64) | v.x;
    }
    __device__ __forceinline__ bool add(const Unit &x) { return add_ovf(a, x.a); }
    __device__ __forceinline__ void store(void *p) const
    {
        *(ulonglong2 *)p = make_ulonglong2((uint64_t)a, (uint64_t)(a >> 64));
    }
    __device__ __forceinline__ Unit xor_shfl(int d) const { Unit r; r.a = shfl_xor(a, d); return r; }
    __device__ __forceinline__ u128 entry(int i) const { return a; }
};

template <typename CT, int UB, int G, int NU, int U, int MB>
__global__ void __launch_bounds__(256, MB) gather_kernel(const __grid_constant__ GatherArgs a)
{
    extern __shared__ int16_t s_map[];
    const int mapn = a.k * a.k * a.Bs;
    for (int i = threadIdx.x; i < mapn; i += blockDim.x) s_map[i] = a.gmap[i];
    __syncthreads();

    typedef Unit<CT, UB> UT;
    constexpr int NG = 32 / G;
    constexpr int EPU = UB / (int)sizeof(CT);  // entries per unit
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, j = lane % G;
    // the lane's units: set and unit within the set
    int uset[NU], usub[NU];
    bool own[NU];
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        const int un = j + i * G;
        own[i] = un < a.ws_units;
        uset[i] = own[i] ? un / a.ups : 0;
        usub[i] = own[i] ? un - uset[i] * a.ups : 0;
    }
    const char *__restrict__ src = (const char *)a.src;
    const int64_t rowb = (int64_t)a.wc_units * UB;
    const int wpb = blockDim.x >> 5;
    bool ovf = false;
    UT acc[NU];

    if ((int)blockIdx.x < a.chunk_blocks) {
        // ---- hub chunks: a warp per chunk
        for (int64_t t = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); t < a.n_chunks;
             t += (int64_t)a.chunk_blocks * wpb) {
            const int64_t v = a.chunk_node[t];
            const int64_t e0 = a.chunk_e0[t], e1 = a.chunk_e1[t];
            const int cv = a.colors[v];
#pragma unroll
            for (int i = 0; i < NU; ++i) acc[i].zero();
            for (int64_t b = e0; b < e1; b += NG * U) {
                UT x[U][NU];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int64_t e = b + q * NG + grp;
                    const bool in = e < e1;
                    const uint32_t u = in ? a.col[e] : 0u;
                    const int cu = in ? (int)a.ecol[e] : cv;
                    const int16_t *gm = s_map + (cv * a.k + cu) * a.Bs;
#pragma unroll
                    for (int i = 0; i < NU; ++i) {
                        const int ss = (in && cu != cv && own[i]) ? gm[uset[i]] : -1;
                        if (ss >= 0) x[q][i].load(src + (int64_t)u * rowb + (int64_t)(ss * a.ups + usub[i]) * UB);
                        else x[q][i].zero();
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q)
#pragma unroll
                    for (int i = 0; i < NU; ++i) ovf |= acc[i].add(x[q][i]);
            }
#pragma unroll
            for (int d = G; d < 32; d <<= 1)
#pragma unroll
                for (int i = 0; i < NU; ++i) ovf |= acc[i].add(acc[i].xor_shfl(d));
            if (grp == 0) {
                // partial row of the chunk, entry-major per hub:
                // [first chunk * Ws + entry * (chunks of the hub) + chunk]
                const int64_t c0 = a.node_chunk0[v];
                const int64_t nch = (a.row_ptr[v + 1] - a.row_ptr[v] + HUB_CHUNK - 1) / HUB_CHUNK;
                CT *out = (CT *)a.partial + c0 * a.Ws + (t - c0);
#pragma unroll
                for (int i = 0; i < NU; ++i)
                    if (own[i])
#pragma unroll
                        for (int w = 0; w < EPU; ++w)
                            out[(int64_t)((j + i * G) * EPU + w) * nch] = acc[i].entry(w);
            }
        }
        if (ovf) atomicOr(a.err, ERR_OVERFLOW);
        return;
    }

    // ---- nodes of degree <= HUB_CHUNK: G lanes per node.  The ids and
    // colours of the next U neighbours are loaded while the rows of the
    // current U are in flight.
    const int64_t nblk = (int64_t)gridDim.x - a.chunk_blocks;
    const int64_t warp0 = ((int64_t)blockIdx.x - a.chunk_blocks) * wpb + (threadIdx.x >> 5);
    for (int64_t base = warp0 * NG; base < a.n_small; base += nblk * wpb * NG) {
        const int64_t idx = base + grp;
        const bool valid = idx < a.n_small;
        const uint4 rec = valid ? a.sched[idx] : make_uint4(0u, 0u, 0u, 0u);
        const int64_t v = rec.x;
        const int64_t e0 = (int64_t)(((uint64_t)rec.z << 32) | rec.y);
        const int d = (int)rec.w;
        const int cv = valid ? (int)a.colors[v] : 0;
        const int dmax = __reduce_max_sync(0xffffffffu, (unsigned)d);
#pragma unroll
        for (int i = 0; i < NU; ++i) acc[i].zero();
        uint32_t nu_[U];
        int ncu[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const bool in = q < d;
            nu_[q] = in ? a.col[e0 + q] : 0u;
            ncu[q] = in ? (int)a.ecol[e0 + q] : cv;
        }
        for (int off = 0; off < dmax; off += U) {
            uint32_t u[U];
            int cu[U];
#pragma unroll
            for (int q = 0; q < U; ++q) { u[q] = nu_[q]; cu[q] = ncu[q]; }
            UT x[U][NU];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int16_t *gm = s_map + (cv * a.k + cu[q]) * a.Bs;
#pragma unroll
                for (int i = 0; i < NU; ++i) {
                    const int ss = (cu[q] != cv && own[i]) ? gm[uset[i]] : -1;
                    if (ss >= 0) x[q][i].load(src + (int64_t)u[q] * rowb + (int64_t)(ss * a.ups + usub[i]) * UB);
                    else x[q][i].zero();
                }
            }
            if (off + U < dmax) {
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const bool in = off + U + q < d;
                    nu_[q] = in ? a.col[e0 + off + U + q] : 0u;
                    ncu[q] = in ? (int)a.ecol[e0 + off + U + q] : cv;
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q)
#pragma unroll
                for (int i = 0; i < NU; ++i) ovf |= acc[i].add(x[q][i]);
        }
        if (valid) {
            char *out = (char *)a.dst + v * (int64_t)a.ws_units * UB;
#pragma unroll
            for (int i = 0; i < NU; ++i)
                if (own[i]) acc[i].store(out + (int64_t)(j + i * G) * UB);
        }
    }
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
}

typedef void (*GatherKernel)(GatherArgs);

// The instantiation for a count width (8 or 16 bytes), unit size, lanes per
// node G, units per lane NU, rows in flight U and blocks-per-SM target MB
// (gather_*.cu); NULL if it is not instantiated.
GatherKernel gather_kernel_ptr(size_t count_bytes, int UB, int G, int NU, int U, int MB);
GatherKernel gather_kernel_ptr_u64_8(int G, int NU, int U, int MB);
GatherKernel gather_kernel_ptr_u64_16(int G, int NU, int U, int MB);
GatherKernel gather_kernel_ptr_u128_16(int G, int NU, int U, int MB);

}  // namespace mc
