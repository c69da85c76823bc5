// build.cu -- the colourful treelet count tables (Section 2.1, Eq. 1).
//
// Per level h the dynamic program runs as two kernels:
//   gather: S_h(v)[T'', C''] = sum_{u ~ v} c_h(u)[T'', C'']      (HBM bound)
//   merge : c_h(v)[T, C] = (1/beta_T) sum_{C' + C'' = C} c_{|T'|}(v)[T', C'] S_{|T''|}(v)[T'', C'']
// with T -> (T', T'') the canonical decomposition (T'' the subtree of the
// root's first child).  Rows are colour-relative: at node v only colour sets
// containing c_v (for c) or avoiding it (for S) are stored, indexed by the
// colex rank of the set with c_v deleted from the palette, so the merge's
// index structure is the same at every node and the gather reads only live
// entries of the neighbour's row.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <tuple>

#include "gather.cuh"

namespace mc {

GatherKernel gather_kernel_ptr(size_t count_bytes, int UB, int G, int NU, int U, int MB)
{
    if (count_bytes == 16) return gather_kernel_ptr_u128_16(G, NU, U, MB);
    return UB == 16 ? gather_kernel_ptr_u64_16(G, NU, U, MB) : gather_kernel_ptr_u64_8(G, NU, U, MB);
}

// The neighbour-sum kernel and its instantiations live in gather.cuh and
// gather_*.cu.
// Sum the chunk partials of each hub into its S row.  The chunk sums of a
// (hub, S entry) pair are contiguous; they become their inclusive prefix
// (the sampler binary-searches it) and the last prefix is the hub's
// neighbour sum.  Any overflowing partial sum means the total overflows too.
// Hubs of at most HUB_SERIAL chunks: a thread per (hub, entry) scans them in
// order (the threads of a warp take consecutive entries of one hub, whose
// chunk sums are adjacent); larger hubs: a warp per (hub, entry), 32 chunks
// per warp scan.

template <typename CT>
__global__ void hub_reduce_small_kernel(CT *__restrict__ partial, CT *__restrict__ dst,
                                        const uint32_t *__restrict__ hub_node,
                                        const int64_t *__restrict__ hub_chunk0, int64_t n_hubs, int Ws, int *err)
{
    bool ovf = false;
    const int64_t total = n_hubs * Ws;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hub = i / Ws;
        const int e = (int)(i - hub * Ws);
        const int64_t c0 = hub_chunk0[hub], nch = hub_chunk0[hub + 1] - c0;
        if (nch > HUB_SERIAL) continue;
        CT *p = partial + c0 * Ws + e * nch;
        CT run = 0;
        for (int64_t c = 0; c < nch; ++c) {
            ovf |= add_ovf(run, p[c]);
            p[c] = run;
        }
        dst[(int64_t)hub_node[hub] * Ws + e] = run;
    }
    if (ovf) atomicOr(err, ERR_OVERFLOW);
}

template <typename CT>
__global__ void hub_reduce_kernel(CT *__restrict__ partial, CT *__restrict__ dst,
                                  const uint32_t *__restrict__ hub_node,
                                  const int64_t *__restrict__ hub_chunk0, const uint32_t *__restrict__ big_hub,
                                  int64_t n_big, int Ws, int *err)
{
    bool ovf = false;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = n_big * Ws;
    for (int64_t i = warp; i < total; i += nwarps) {
        const int64_t bi = i / Ws;
        const int e = (int)(i - bi * Ws);
        const int64_t hub = big_hub[bi];
        const int64_t c0 = hub_chunk0[hub], nch = hub_chunk0[hub + 1] - c0;
        CT *p = partial + c0 * Ws + e * nch;
        CT carry = 0;
        for (int64_t b = 0; b < nch; b += 32) {
            const int64_t c = b + lane;
            CT x = c < nch ? p[c] : (CT)0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const CT y = shfl_up(x, d);
                if (lane >= d) ovf |= add_ovf(x, y);
            }
            ovf |= add_ovf(x, carry);
            if (c < nch) p[c] = x;
            carry = shfl(x, 31);
        }
        if (lane == 0) dst[(int64_t)hub_node[hub] * Ws + e] = carry;
    }
    if (ovf) atomicOr(err, ERR_OVERFLOW);
}

// ---------------------------------------------------------------------------
// merge of level h: one thread per (node, output entry).  Output o of level
// h carries (|T'|, |T''|, beta, #terms) and a list of (index into the
// c_{|T'|} row, index into the S_{|T''|} row) pairs, one per split of the
// colour set; c_1 is the constant 1.
// ---------------------------------------------------------------------------
struct MergeArgs {
    const void *c[MAXK + 1];
    const void *S[MAXK + 1];
    int Wc[MAXK + 1], Ws[MAXK + 1];
    ExactDiv div[MAXK + 1];
    const int32_t *info, *off;
    const uint32_t *terms;
    void *out;
    int64_t n;
    int W, Bc, R;                     // row width, colour sets and shapes of the level
    const MergeLevel *program;        // host copy of the program (schedule planning only)
    const uint8_t *zero_root_colors;  // set: only colour-0 nodes get counts
    int *err;
};

template <typename CT, int MINB>
__global__ void __launch_bounds__(256, MINB) merge_kernel(const __grid_constant__ MergeArgs a)
{
    bool ovf = false, inexact = false;
    const int64_t total = a.n * a.W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        // node and output entry; 32-bit division when the level fits 2^32
        // entries.  Threads walk a row in (shape, set) order, so the threads
        // of a warp mostly share one shape and one program length, and write
        // entry (set, shape) at its set-major position.
        const int64_t v = total <= 0xffffffffll ? (int64_t)((uint32_t)t / (uint32_t)a.W) : t / a.W;
        const int q = (int)(t - v * a.W);
        const int sh = q / a.Bc;
        const int o = (q - sh * a.Bc) * a.R + sh;
        if (a.zero_root_colors && a.zero_root_colors[v] != 0) {
            ((CT *)a.out)[v * a.W + o] = 0;
            continue;
        }
        const int info = a.info[o];
        const int h1 = info & 15, h2 = (info >> 4) & 15, beta = (info >> 8) & 255, nt = info >> 16;
        const uint32_t *term = a.terms + a.off[o];
        const CT *B = (const CT *)a.S[h2] + v * a.Ws[h2];
        CT sum = 0;
        if (h1 == 1) {
            for (int i = 0; i < nt; ++i) ovf |= add_ovf(sum, B[term[i] >> 16]);
        } else {
            const CT *A = (const CT *)a.c[h1] + v * a.Wc[h1];
            for (int i = 0; i < nt; ++i) {
                const uint32_t tm = term[i];
                CT p;
                ovf |= mul_ovf(A[tm & 0xffffu], B[tm >> 16], p);
                ovf |= add_ovf(sum, p);
            }
        }
        CT qt;
        if (!exact_div(sum, a.div[beta], qt)) inexact = true;
        ((CT *)a.out)[v * a.W + o] = qt;
    }
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (inexact) atomicOr(a.err, ERR_INEXACT);
}

// The merge with its operands streamed through shared memory: a block takes
// tiles of NB consecutive nodes; while it computes the outputs of one tile
// from one buffer, cp.async copies the next tile's rows (every lower level
// the program reads; rows of consecutive nodes are contiguous) into the
// other, 16 bytes per copy.  Waiting is cp.async.wait_group on the thread's
// own copies, followed by a block barrier.
struct MergeStage {
    int nlev;
    int is_s[2 * MAXK];
    int lev[2 * MAXK];
    int off[2 * MAXK];        // offset of the level's NB rows inside one buffer, in counts
    int soff_c[MAXK + 1];     // the same per c level (-1: not staged)
    int soff_s[MAXK + 1];
    int NB;
    int buf;                  // counts per buffer
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename CT>
__device__ __forceinline__ void merge_stage_copy(const MergeArgs &a, const MergeStage &st, int64_t tile, CT *buf)
{
    const int64_t v0 = tile * st.NB;
    if (v0 >= a.n) return;
    const int nv = (int)min((int64_t)st.NB, a.n - v0);
    for (int l = 0; l < st.nlev; ++l) {
        const int h = st.lev[l];
        const int W = st.is_s[l] ? a.Ws[h] : a.Wc[h];
        const char *g = (const char *)((const CT *)(st.is_s[l] ? a.S[h] : a.c[h]) + v0 * W);
        char *d = (char *)(buf + st.off[l]);
        const int chunks = (int)(((int64_t)nv * W * (int64_t)sizeof(CT)) >> 4);
        for (int i = threadIdx.x; i < chunks; i += blockDim.x) cp_async16(d + 16 * i, g + 16 * i);
    }
}

template <typename CT>
__global__ void __launch_bounds__(256) merge_pipe_kernel(const __grid_constant__ MergeArgs a,
                                                         const __grid_constant__ MergeStage st)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    CT *bufs = (CT *)s_raw;
    bool ovf = false, inexact = false;
    const int64_t ntiles = (a.n + st.NB - 1) / st.NB;
    int64_t tile = blockIdx.x;
    merge_stage_copy<CT>(a, st, tile, bufs);
    cp_async_commit();
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        CT *cur = bufs + (int64_t)(it & 1) * st.buf;
        merge_stage_copy<CT>(a, st, tile + gridDim.x, bufs + (int64_t)((it + 1) & 1) * st.buf);
        cp_async_commit();
        cp_async_wait1();   // this thread's copies of `tile` have landed
        __syncthreads();    // and every other thread's
        const int64_t v0 = tile * st.NB;
        const int nv = (int)min((int64_t)st.NB, a.n - v0);
        const int nout = nv * a.W;
        for (int t = threadIdx.x; t < nout; t += blockDim.x) {
            const int vl = t / a.W;
            const int q = t - vl * a.W;
            const int sh = q / a.Bc;
            const int o = (q - sh * a.Bc) * a.R + sh;
            const int64_t v = v0 + vl;
            CT *dst = (CT *)a.out + v * a.W + o;
            if (a.zero_root_colors && a.zero_root_colors[v] != 0) {
                *dst = 0;
                continue;
            }
            const int info = a.info[o];
            const int h1 = info & 15, h2 = (info >> 4) & 15, beta = (info >> 8) & 255, nt = info >> 16;
            const uint32_t *term = a.terms + a.off[o];
            CT sum = 0;
            if (nt > 0) {
                const CT *B = cur + st.soff_s[h2] + vl * a.Ws[h2];
                if (h1 == 1) {
                    for (int i = 0; i < nt; ++i) ovf |= add_ovf(sum, B[term[i] >> 16]);
                } else {
                    const CT *A = cur + st.soff_c[h1] + vl * a.Wc[h1];
                    for (int i = 0; i < nt; ++i) {
                        const uint32_t tm = term[i];
                        CT p;
                        ovf |= mul_ovf(A[tm & 0xffffu], B[tm >> 16], p);
                        ovf |= add_ovf(sum, p);
                    }
                }
            }
            CT qt;
            if (!exact_div(sum, a.div[beta], qt)) inexact = true;
            *dst = qt;
        }
        __syncthreads();    // the buffer is free for the copy two tiles ahead
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (inexact) atomicOr(a.err, ERR_INEXACT);
}

// The same merge with a thread per node walking all W outputs of its row in
// (shape, set) order: every lane of a warp runs the same output program at
// the same time (no divergence; the program's loads are uniform), reading
// its own node's rows.
template <typename CT, int MINB>
__global__ void __launch_bounds__(256, MINB) merge_node_kernel(const __grid_constant__ MergeArgs a)
{
    bool ovf = false, inexact = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.n; v += (int64_t)gridDim.x * blockDim.x) {
        CT *row = (CT *)a.out + v * a.W;
        const bool zero = a.zero_root_colors && a.zero_root_colors[v] != 0;
        for (int sh = 0; sh < a.R; ++sh)
            for (int rho = 0; rho < a.Bc; ++rho) {
                const int o = rho * a.R + sh;
                if (zero) { row[o] = 0; continue; }
                const int info = a.info[o];
                const int h1 = info & 15, h2 = (info >> 4) & 15, beta = (info >> 8) & 255, nt = info >> 16;
                const uint32_t *term = a.terms + a.off[o];
                const CT *B = (const CT *)a.S[h2] + v * a.Ws[h2];
                CT sum = 0;
                if (h1 == 1) {
                    for (int i = 0; i < nt; ++i) ovf |= add_ovf(sum, B[term[i] >> 16]);
                } else {
                    const CT *A = (const CT *)a.c[h1] + v * a.Wc[h1];
                    for (int i = 0; i < nt; ++i) {
                        const uint32_t tm = term[i];
                        CT p;
                        ovf |= mul_ovf(A[tm & 0xffffu], B[tm >> 16], p);
                        ovf |= add_ovf(sum, p);
                    }
                }
                CT qt;
                if (!exact_div(sum, a.div[beta], qt)) inexact = true;
                row[o] = qt;
            }
    }
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (inexact) atomicOr(a.err, ERR_INEXACT);
}

// ---------------------------------------------------------------------------
// per-node totals of a level over a set of shapes, and an inclusive u128
// prefix over the nodes (the cumulative counts of Section 3.2.1, taken over
// nodes for the root draw).
// ---------------------------------------------------------------------------
template <typename CT, int G>
__global__ void __launch_bounds__(256) row_totals_kernel(const CT *__restrict__ c, int64_t n, int W, int R,
                                                         uint64_t allow0, uint64_t allow1,
                                                         u128 *__restrict__ tot, int *err)
{
    // groups of G lanes per node, 32/G nodes per warp
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, j = lane % G;
    constexpr int NG = 32 / G;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool ovf = false;
    for (int64_t v0 = warp * NG; v0 < n; v0 += nwarps * NG) {
        const int64_t v = v0 + grp;
        u128 s = 0;
        if (v < n)
            for (int eb = j; eb < W; eb += 8 * G) {  // up to 8 loads in flight per lane
                CT x[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int e = eb + i * G;
                    const int sh = e % R;  // set-major row: entry e is (set e / R, shape e % R)
                    const bool ok = e < W && (sh < 64 ? (allow0 >> sh) & 1 : (allow1 >> (sh - 64)) & 1);
                    x[i] = ok ? c[v * W + e] : (CT)0;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) ovf |= add_ovf(s, widen(x[i]));
            }
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const u128 o = shfl_xor(s, d);
            ovf |= add_ovf(s, o);
        }
        if (j == 0 && v < n) tot[v] = s;
    }
    if (ovf) atomicOr(err, ERR_OVERFLOW);
}

// The rooted shapes of each unrooted treelet at one level: treelet j owns
// shape[off[j] .. off[j + 1]).
struct TreeletShapes {
    int16_t off[32];
    uint8_t shape[128];
};

// Per node and unrooted treelet T_j: the sum of the node's level-h counts
// over the rooted shapes of T_j and all colour sets, tot[j * n + v].  One
// thread per (node, treelet), treelet fastest, so a warp reads a few whole
// rows.  Overflow of a sum is flagged.
template <typename CT>
__global__ void __launch_bounds__(256) treelet_totals_kernel(const CT *__restrict__ c, int64_t n, int W, int R, int Bc,
                                                             int nu, const __grid_constant__ TreeletShapes ts,
                                                             u128 *__restrict__ tot, int *err)
{
    bool ovf = false;
    const int64_t total = n * nu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / nu;
        const int j = (int)(i - v * nu);
        const CT *row = c + v * W;
        u128 s = 0;
        for (int q = ts.off[j]; q < ts.off[j + 1]; ++q) {
            const int sh = ts.shape[q];
            for (int b = 0; b < Bc; ++b) ovf |= add_ovf(s, widen(row[b * R + sh]));
        }
        tot[(int64_t)j * n + v] = s;
    }
    if (ovf) atomicOr(err, ERR_OVERFLOW);
}

constexpr int SCAN_THREADS = 512, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ u128 block_exclusive_scan(u128 x, u128 *smem, u128 &block_total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u128 inc = warp_inclusive_scan(x);
    if (lane == 31) smem[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        u128 y = lane < nw ? smem[lane] : 0;
        y = warp_inclusive_scan(y);
        if (lane < nw) smem[lane] = y;
    }
    __syncthreads();
    const u128 before = w > 0 ? smem[w - 1] : 0;
    block_total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + inc - x;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles_kernel(const u128 *__restrict__ x, int64_t n,
                                                                  u128 *__restrict__ tile_sum, int *err)
{
    __shared__ u128 smem[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    u128 s = 0;
    bool ovf = false;
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) ovf |= add_ovf(s, x[base + i]);
    u128 tot;
    const u128 ex = block_exclusive_scan(s, smem, tot);
    // the block total is exact iff no prefix wrapped
    if (ex + s < ex) ovf = true;
    if (threadIdx.x == blockDim.x - 1) tile_sum[blockIdx.x] = tot;
    if (ovf) atomicOr(err, ERR_OVERFLOW);
}

__global__ void __launch_bounds__(1024) scan_tile_sums_kernel(u128 *tile_sum, int64_t ntiles, int *err)
{
    __shared__ u128 smem[32];
    u128 carry = 0;
    bool ovf = false;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const u128 x = i < ntiles ? tile_sum[i] : 0;
        u128 tot;
        const u128 ex = block_exclusive_scan(x, smem, tot);
        const u128 before = carry + ex;
        if (before < carry || before + x < before) ovf = true;
        if (i < ntiles) tile_sum[i] = before;  // exclusive
        const u128 nc = carry + tot;
        if (nc < carry) ovf = true;
        carry = nc;
    }
    if (ovf) atomicOr(err, ERR_OVERFLOW);
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_apply_kernel(u128 *__restrict__ x, int64_t n,
                                                                  const u128 *__restrict__ tile_ex)
{
    __shared__ u128 smem[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    u128 v[SCAN_ITEMS];
    u128 s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? x[base + i] : 0;
        s += v[i];
    }
    u128 tot;
    u128 run = block_exclusive_scan(s, smem, tot) + tile_ex[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        run += v[i];
        if (base + i < n) x[base + i] = run;
    }
}

// Colour of every edge's far end, so that neighbour loops read colours
// contiguously instead of one random byte per neighbour.
__global__ void edge_colours_kernel(const uint32_t *__restrict__ col, const uint8_t *__restrict__ colors,
                                    int64_t nnz, uint8_t *__restrict__ ecol)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        ecol[e] = colors[col[e]];
}

// Colour blocks: every node's neighbour list stably partitioned by the
// neighbours' colours (scol), with the block starts (coff, k+1 per node).
// Nodes of degree <= HUB_CHUNK: one thread each, per-colour counts and
// cursors packed one byte per colour.
// The per-colour counts are also the level-1 neighbour sums S_1(v)[{a}]
// (c of a single node is 1 at its own colour), written here too.
template <typename CT>
__global__ void colour_blocks_kernel(const int64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                                     const uint8_t *__restrict__ ecol, const uint8_t *__restrict__ colors,
                                     int64_t n, int k, uint32_t *__restrict__ scol, int32_t *__restrict__ coff,
                                     CT *__restrict__ S1)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        if (e1 - e0 > HUB_CHUNK) continue;
        uint64_t cnt = 0;
        for (int64_t e = e0; e < e1; ++e) cnt += 1ull << (8 * ecol[e]);
        uint64_t cur = 0;  // exclusive prefix of the counts, one byte per colour
        uint32_t run = 0;
        for (int a = 0; a < k; ++a) {
            coff[v * (k + 1) + a] = (int32_t)run;
            cur |= (uint64_t)run << (8 * a);
            run += (uint32_t)((cnt >> (8 * a)) & 0xffu);
        }
        coff[v * (k + 1) + k] = (int32_t)run;
        const int cv = colors[v];
        for (int a = 0; a < k - 1; ++a) {
            const int abs_a = a < cv ? a : a + 1;
            S1[v * (k - 1) + a] = (CT)((cnt >> (8 * abs_a)) & 0xffu);
        }
        for (int64_t e = e0; e < e1; ++e) {
            const int c = ecol[e];
            const uint32_t pos = (uint32_t)((cur >> (8 * c)) & 0xffu);
            cur += 1ull << (8 * c);
            scol[e0 + pos] = col[e];
        }
    }
}

// The same for hubs, one warp per hub: per-colour ballots give each edge's
// rank among the earlier edges of its colour.
// Hubs: the same, spread over their 64-neighbour chunks so no warp walks a
// whole hub.  (1) per chunk, per-colour counts; (2) per hub, the exclusive
// prefix of those counts over its chunks (each chunk's start inside every
// colour block), the block starts and S_1; (3) per chunk, the scatter.
static_assert(HUB_CHUNK <= 64, "hub chunk kernels read two 32-edge rounds per chunk");

__global__ void hub_chunk_counts_kernel(const uint8_t *__restrict__ ecol, const int64_t *__restrict__ chunk_e0,
                                        const int64_t *__restrict__ chunk_e1, int64_t n_chunks, int k,
                                        uint32_t *__restrict__ ccnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp; c < n_chunks; c += nwarps) {
        const int64_t e0 = chunk_e0[c], e1 = chunk_e1[c];
        const int c0 = e0 + lane < e1 ? (int)ecol[e0 + lane] : -1;
        const int c1 = e0 + 32 + lane < e1 ? (int)ecol[e0 + 32 + lane] : -1;
        uint32_t mine = 0;
#pragma unroll
        for (int a = 0; a < MAXK; ++a)
            if (a < k) {
                const uint32_t x = __popc(__ballot_sync(0xffffffffu, c0 == a)) +
                                   __popc(__ballot_sync(0xffffffffu, c1 == a));
                if (lane == a) mine = x;
            }
        if (lane < k) ccnt[c * k + lane] = mine;
    }
}

template <typename CT>
__global__ void hub_chunk_prefix_kernel(const uint8_t *__restrict__ colors, const uint32_t *__restrict__ hub_node,
                                        const int64_t *__restrict__ hub_chunk0, int64_t n_hubs, int k,
                                        uint32_t *__restrict__ ccnt, int32_t *__restrict__ coff,
                                        CT *__restrict__ S1)
{
    // one warp per hub: lanes take 32 chunks at a time; a warp scan per
    // colour turns the counts, in place, into each chunk's start inside that
    // colour's block
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t hb = warp; hb < n_hubs; hb += nwarps) {
        const int64_t v = hub_node[hb];
        const int64_t c0 = hub_chunk0[hb], c1 = hub_chunk0[hb + 1];
        uint32_t tot[MAXK];
#pragma unroll
        for (int a = 0; a < MAXK; ++a) tot[a] = 0;
        for (int64_t b = c0; b < c1; b += 32) {
            const int64_t c = b + lane;
#pragma unroll
            for (int a = 0; a < MAXK; ++a)
                if (a < k) {
                    const uint32_t x = c < c1 ? ccnt[c * k + a] : 0u;
                    uint32_t inc = x;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
                        if (lane >= d) inc += y;
                    }
                    if (c < c1) ccnt[c * k + a] = tot[a] + inc - x;
                    tot[a] += __shfl_sync(0xffffffffu, inc, 31);
                }
        }
        if (lane == 0) {
            uint32_t run = 0;
#pragma unroll
            for (int a = 0; a < MAXK; ++a)
                if (a < k) {
                    coff[v * (k + 1) + a] = (int32_t)run;
                    run += tot[a];
                }
            coff[v * (k + 1) + k] = (int32_t)run;
            const int cv = colors[v];
#pragma unroll
            for (int a = 0; a < MAXK - 1; ++a)
                if (a < k - 1) S1[v * (k - 1) + a] = (CT)tot[a < cv ? a : a + 1];
        }
    }
}

__global__ void hub_chunk_scatter_kernel(const uint32_t *__restrict__ col, const uint8_t *__restrict__ ecol,
                                         const int64_t *__restrict__ row_ptr,
                                         const uint32_t *__restrict__ chunk_node,
                                         const int64_t *__restrict__ chunk_e0, const int64_t *__restrict__ chunk_e1,
                                         int64_t n_chunks, int k, const uint32_t *__restrict__ cstart,
                                         const int32_t *__restrict__ coff, uint32_t *__restrict__ scol)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp; c < n_chunks; c += nwarps) {
        const int64_t v = chunk_node[c];
        const int64_t base = row_ptr[v];
        const int64_t e0 = chunk_e0[c], e1 = chunk_e1[c];
        int cc[2];
        uint32_t uu[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int64_t e = e0 + 32 * r + lane;
            cc[r] = e < e1 ? (int)ecol[e] : -1;
            uu[r] = e < e1 ? col[e] : 0u;
        }
        uint32_t pos[MAXK];
#pragma unroll
        for (int a = 0; a < MAXK; ++a)
            pos[a] = a < k ? (uint32_t)coff[v * (k + 1) + a] + cstart[c * k + a] : 0u;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            uint32_t my = 0;
#pragma unroll
            for (int a = 0; a < MAXK; ++a)
                if (a < k) {
                    const unsigned m = __ballot_sync(0xffffffffu, cc[r] == a);
                    if (cc[r] == a) my = pos[a] + __popc(m & lt);
                    pos[a] += __popc(m);
                }
            if (cc[r] >= 0) scol[base + my] = uu[r];
        }
    }
}

// Root-search buckets: X in [0, R) falls in bucket b = floor(X / D), D =
// ceil(R / nb); start[b] is the first node whose inclusive prefix exceeds
// b * D, so the node drawn for X lies in [start[b], start[b + 1]].
__global__ void bucket_width_kernel(const u128 *prefix, int64_t n, int64_t nb, u128 *D)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const u128 R = n > 0 ? prefix[n - 1] : 0;
        u128 d = R / (u128)nb + ((R % (u128)nb) != 0 ? 1 : 0);
        *D = d ? d : 1;
    }
}

__global__ void bucket_kernel(const u128 *__restrict__ prefix, int64_t n, int64_t nb, const u128 *Dp,
                              uint32_t *__restrict__ start)
{
    const u128 D = *Dp;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= nb;
         b += (int64_t)gridDim.x * blockDim.x) {
        const u128 X = (u128)b * D;
        int64_t lo = 0, hi = n;  // first v with prefix[v] > X, else n - 1
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (prefix[mid] > X) hi = mid; else lo = mid + 1;
        }
        start[b] = (uint32_t)(lo < n ? lo : n - 1);
    }
}

void build_buckets(const u128 *prefix, int64_t n, int64_t nb, u128 *dD, uint32_t *start, cudaStream_t s)
{
    if (n <= 0) return;
    MC_LAUNCH("bucket_width", s, bucket_width_kernel<<<1, 32, 0, s>>>(prefix, n, nb, dD));
    MC_LAUNCH("buckets", s, bucket_kernel<<<grid_for(nb + 1, 256), 256, 0, s>>>(prefix, n, nb, dD, start));
}

int64_t bucket_count(int64_t n) { return std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)1 << 22)); }

// A colour >= k is reported and replaced by 0 in the tables' own copy, so
// the kernels after this one never index past a colour's slot; the build
// then fails when its error flags are read.
__global__ void check_colours_kernel(uint8_t *colors, int64_t n, int k, int *err)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (colors[v] >= k) {
            atomicOr(err, ERR_COLOUR);
            colors[v] = 0;
        }
}

__global__ void fill_ones_kernel(void *dst, int64_t n, int bytes)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (bytes == 8) ((uint64_t *)dst)[i] = 1;
        else ((u128 *)dst)[i] = 1;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int64_t scan_tiles(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// the scan with a caller-provided tile-sum buffer of scan_tiles(n) entries
static void inclusive_scan_u128_buf(u128 *x, int64_t n, int *err, u128 *ts, cudaStream_t s)
{
    if (n <= 0) return;
    const int64_t ntiles = scan_tiles(n);
    MC_LAUNCH("scan_tiles", s, scan_tiles_kernel<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(x, n, ts, err));
    MC_LAUNCH("scan_tile_sums", s, scan_tile_sums_kernel<<<1, 1024, 0, s>>>(ts, ntiles, err));
    MC_LAUNCH("scan_apply", s, scan_apply_kernel<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(x, n, ts));
}

void inclusive_scan_u128(u128 *x, int64_t n, int *err, Arena &scratch, cudaStream_t s)
{
    if (n <= 0) return;
    inclusive_scan_u128_buf(x, n, err, scratch.get<u128>((size_t)scan_tiles(n)), s);
}

ExactDiv make_div(int beta)
{
    ExactDiv d{};
    int t = 0;
    while (!((beta >> t) & 1)) ++t;
    const uint64_t odd = (uint64_t)(beta >> t);
    // Newton iteration for the inverse of an odd number modulo 2^64 / 2^128
    uint64_t inv = odd;  // correct to 3 bits
    for (int i = 0; i < 6; ++i) inv *= 2 - odd * inv;
    u128 inv2 = inv;
    for (int i = 0; i < 2; ++i) inv2 *= (u128)2 - (u128)odd * inv2;
    d.shift = t;
    d.inv64 = inv;
    d.inv128 = inv2;
    d.qmax64 = ~0ull / odd;
    d.qmax128 = (~(u128)0) / (u128)odd;
    return d;
}

template <typename CT> size_t bytes_of() { return sizeof(CT); }

template <typename CT>
static void launch_row_totals_t(const CT *c, int64_t n, int W, int R, uint64_t allow0, uint64_t allow1, u128 *tot,
                                int *err, cudaStream_t s)
{
    int G = 1;  // lanes per node: each covers up to 8 entries
    while (G * 8 < W && G < 32) G <<= 1;
    const int grid = grid_for((n * G + 31) / 32 * 32, 256);
    switch (G) {
    case 1: MC_LAUNCH("row_totals", s, row_totals_kernel<CT, 1><<<grid, 256, 0, s>>>(c, n, W, R, allow0, allow1, tot, err)); break;
    case 2: MC_LAUNCH("row_totals", s, row_totals_kernel<CT, 2><<<grid, 256, 0, s>>>(c, n, W, R, allow0, allow1, tot, err)); break;
    case 4: MC_LAUNCH("row_totals", s, row_totals_kernel<CT, 4><<<grid, 256, 0, s>>>(c, n, W, R, allow0, allow1, tot, err)); break;
    case 8: MC_LAUNCH("row_totals", s, row_totals_kernel<CT, 8><<<grid, 256, 0, s>>>(c, n, W, R, allow0, allow1, tot, err)); break;
    case 16: MC_LAUNCH("row_totals", s, row_totals_kernel<CT, 16><<<grid, 256, 0, s>>>(c, n, W, R, allow0, allow1, tot, err)); break;
    default: MC_LAUNCH("row_totals", s, row_totals_kernel<CT, 32><<<grid, 256, 0, s>>>(c, n, W, R, allow0, allow1, tot, err)); break;
    }
}

void launch_row_totals(const mc_tables *t, int h, uint64_t allow0, uint64_t allow1, u128 *tot, int *err,
                       cudaStream_t s)
{
    const int64_t n = t->g->n;
    if (n == 0) return;
    if (t->packed) {
        launch_packed_row_totals(t, h, allow0, allow1, tot, err, s);
        return;
    }
    const int W = t->geo.Wc[h], R = shape_catalog().r[h];
    if (t->bits == 64)
        launch_row_totals_t<uint64_t>((const uint64_t *)t->c[h], n, W, R, allow0, allow1, tot, err, s);
    else
        launch_row_totals_t<u128>((const u128 *)t->c[h], n, W, R, allow0, allow1, tot, err, s);
}

// Dense tables: tot[j * n + v] for every unrooted treelet j of level h in
// one pass over the level's c rows.
void launch_treelet_totals(const mc_tables *t, int h, u128 *tot, int *err, cudaStream_t s)
{
    const int64_t n = t->g->n;
    const ShapeCatalog &cat = shape_catalog();
    const int nu = cat.n_unrooted[h], R = cat.r[h];
    if (n == 0 || nu == 0) return;
    MC_REQUIRE(!t->packed, "treelet totals read dense tables");
    TreeletShapes ts{};
    int q = 0;
    for (int j = 0; j < nu; ++j) {
        ts.off[j] = (int16_t)q;
        for (int i = 0; i < R; ++i)
            if (cat.shapes[cat.gid(h, i)].unrooted == j) ts.shape[q++] = (uint8_t)i;
    }
    ts.off[nu] = (int16_t)q;
    const int W = t->geo.Wc[h], Bc = t->geo.Bc[h];
    const int grid = grid_for(n * nu, 256);
    if (t->bits == 64)
        MC_LAUNCH("treelet_totals", s, treelet_totals_kernel<uint64_t><<<grid, 256, 0, s>>>(
                                           (const uint64_t *)t->c[h], n, W, R, Bc, nu, ts, tot, err));
    else
        MC_LAUNCH("treelet_totals", s, treelet_totals_kernel<u128><<<grid, 256, 0, s>>>(
                                           (const u128 *)t->c[h], n, W, R, Bc, nu, ts, tot, err));
}

static const char *const kGatherName[MAXK + 1] = {"gather_h0", "gather_h1", "gather_h2", "gather_h3",
                                                  "gather_h4", "gather_h5", "gather_h6", "gather_h7",
                                                  "gather_h8"};
static const char *const kMergeName[MAXK + 1] = {"merge_h0", "merge_h1", "merge_h2", "merge_h3", "merge_h4",
                                                 "merge_h5", "merge_h6", "merge_h7", "merge_h8"};

static int rows_in_flight(int NU) { return NU >= 16 ? 1 : NU >= 8 ? 2 : NU >= 4 ? 4 : 8; }

// Schedule candidates of the neighbour sums (the autotuner's choices), on
// G0 lanes per node (the smallest power of two covering the row's units, at
// most 32) and NU0 units per lane, with R0 = the standard rows in flight:
//   0: R0 rows in flight, no register cap
//   1: R0 / 2,  2: R0 / 4 (fewer registers, more warps per SM)
//   3: R0 / 2 with at most 40 registers (6 blocks of 256 per SM)
//   4: R0 / 4 with at most 32 registers (8 blocks of 256 per SM)
//   5: one row in flight, 8 blocks per SM
//   6: G0 / 2 lanes per node with two units each (twice the nodes per warp),
//      a quarter of their rows in flight, 8 blocks per SM (2 <= G0 <= 16)
constexpr int GATHER_CANDIDATES = 7;

template <typename CT, int UB>
static bool launch_gather_ub(const GatherArgs &ga, int h, int cand, cudaStream_t s)
{
    int G = 1;
    while (G < ga.ws_units && G < 32) G <<= 1;
    int NU = 1;
    while (NU * 32 < ga.ws_units) NU <<= 1;
    if (NU > 16) throw Error(MC_E_INTERNAL, "gather: S row too wide");
    const int R0 = rows_in_flight(NU);
    int U = R0, MB = 1;
    switch (cand) {
    case 0: break;
    case 1: U = std::max(1, R0 / 2); break;
    case 2: U = std::max(1, R0 / 4); break;
    case 3: U = std::max(1, R0 / 2); MB = 6; break;
    case 4: U = std::max(1, R0 / 4); MB = 8; break;
    case 5: U = 1; MB = 8; break;
    case 6:
        if (G < 2 || G > 16) return false;
        G /= 2;
        NU *= 2;
        U = std::max(1, rows_in_flight(NU) / 4);
        MB = 8;
        break;
    default: return false;
    }
    auto kern = gather_kernel_ptr(sizeof(CT), UB, G, NU, U, MB);
    if (!kern) return false;
    const int NG = 32 / G;
    const int wpb = 256 / 32;
    GatherArgs g2 = ga;
    const int64_t cap = (int64_t)sm_count() * 32;
    g2.chunk_blocks = (int)std::min<int64_t>((ga.n_chunks + wpb - 1) / wpb, cap);
    const int64_t node_blocks = std::max<int64_t>(1, std::min<int64_t>((ga.n_small + NG * wpb - 1) / (NG * wpb), cap));
    const int grid = (int)(g2.chunk_blocks + node_blocks);
    const size_t smem = (size_t)ga.k * ga.k * ga.Bs * sizeof(int16_t);
    MC_LAUNCH(kGatherName[h], s, kern<<<grid, 256, smem, s>>>(g2));
    return true;
}

template <typename CT> static bool launch_gather(GatherArgs &ga, int r, int h, int cand, cudaStream_t s)
{
    const int B = (int)sizeof(CT);
    const int UB = (r * B) % 16 == 0 ? 16 : 8;  // a unit never straddles two colour sets
    ga.ups = r * B / UB;
    ga.wc_units = ga.Wc * B / UB;
    ga.ws_units = ga.Ws * B / UB;
    if (UB == 16) return launch_gather_ub<CT, 16>(ga, h, cand, s);
    return launch_gather_ub<uint64_t, 8>(ga, h, cand, s);
}

// The pipelined merge's staging plan for level h: the lower levels its
// program reads, NB nodes per tile with two tiles of at most 96 KB of rows
// per block; false when rows cannot be copied in 16-byte pieces.
template <typename CT>
static bool merge_stage_plan(const MergeArgs &ma, const MergeLevel &M, int h, MergeStage &st)
{
    bool use_c[MAXK + 1] = {false}, use_s[MAXK + 1] = {false};
    for (int32_t info : M.info) {
        if ((info >> 16) == 0) continue;
        const int h1 = info & 15, h2 = (info >> 4) & 15;
        if (h1 >= 2) use_c[h1] = true;
        use_s[h2] = true;
    }
    int per_node = 0;
    for (int x = 1; x < h; ++x) per_node += (use_c[x] ? ma.Wc[x] : 0) + (use_s[x] ? ma.Ws[x] : 0);
    if (per_node == 0) return false;
    const int cb = (int)sizeof(CT);
    int NB = (int)std::min<int64_t>(64, (48 * 1024) / ((int64_t)per_node * cb));
    if (cb == 8) NB &= ~1;  // u64 rows: an even count of rows per level is 16-byte aligned
    if (NB < 1) return false;
    st = MergeStage{};
    st.NB = NB;
    for (int x = 0; x <= MAXK; ++x) st.soff_c[x] = st.soff_s[x] = -1;
    int off = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int x = 1; x < h; ++x) {
            if (!(pass ? use_s[x] : use_c[x])) continue;
            const int W = pass ? ma.Ws[x] : ma.Wc[x];
            st.is_s[st.nlev] = pass;
            st.lev[st.nlev] = x;
            st.off[st.nlev] = off;
            (pass ? st.soff_s : st.soff_c)[x] = off;
            off += NB * W;
            ++st.nlev;
        }
    st.buf = off;
    return true;
}

// Merge candidates: a thread per output entry with occupancy targets of 1
// (no register cap), 6 and 8 blocks of 256 threads per SM; a thread per node
// (all of its outputs) at 6 and 8 blocks per SM; the pipelined merge through
// shared memory.
constexpr int MERGE_CANDIDATES = 6;

template <typename CT> static bool launch_merge(const MergeArgs &ma, int h, int cand, cudaStream_t s)
{
    const int grid = grid_for(ma.n * ma.W, 256);
    const int gnode = grid_for(ma.n, 256);
    switch (cand) {
    case 0: MC_LAUNCH(kMergeName[h], s, merge_kernel<CT, 1><<<grid, 256, 0, s>>>(ma)); return true;
    case 1: MC_LAUNCH(kMergeName[h], s, merge_kernel<CT, 6><<<grid, 256, 0, s>>>(ma)); return true;
    case 2: MC_LAUNCH(kMergeName[h], s, merge_kernel<CT, 8><<<grid, 256, 0, s>>>(ma)); return true;
    case 3: MC_LAUNCH(kMergeName[h], s, merge_node_kernel<CT, 6><<<gnode, 256, 0, s>>>(ma)); return true;
    case 4: MC_LAUNCH(kMergeName[h], s, merge_node_kernel<CT, 8><<<gnode, 256, 0, s>>>(ma)); return true;
    case 5: {
        MergeStage st;
        if (!ma.program || !merge_stage_plan<CT>(ma, *ma.program, h, st)) return false;
        // the last partial tile of u64 rows may be an odd count: 16-byte
        // copies need even tiles throughout
        if (sizeof(CT) == 8 && (ma.n % st.NB) != 0 && ((ma.n % st.NB) & 1)) return false;
        const size_t smem = 2 * (size_t)st.buf * sizeof(CT);
        if (smem > 48 * 1024)
            MC_CUDA(cudaFuncSetAttribute(merge_pipe_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t ntiles = (ma.n + st.NB - 1) / st.NB;
        const int g = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * 4);
        MC_LAUNCH(kMergeName[h], s, merge_pipe_kernel<CT><<<g, 256, smem, s>>>(ma, st));
        return true;
    }
    default: return false;
    }
}

// ---------------------------------------------------------------------------
// Autotuner: the schedule of each (kernel, k, count width, level, graph
// shape) is chosen by timing every candidate once on the first build that
// meets it (the candidates compute identical tables, so which one runs does
// not change any result).  The graph's shape is reduced to a degree bucket:
// log2 n, log2 of the average degree in half steps, log2 of the largest
// degree.  Choices can be loaded from and appended to a cache file
// (mc_autotune, or the MC_AUTOTUNE_CACHE environment variable).
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
    int kind, k, bits, h, logn, logdeg, loghub;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(kind, k, bits, h, logn, logdeg, loghub) <
               std::tie(o.kind, o.k, o.bits, o.h, o.logn, o.logdeg, o.loghub);
    }
};
struct TuneState {
    std::mutex mu;
    std::map<TuneKey, int> choice;
    std::set<TuneKey> retuned;  // mode 2: keys tuned again in this process
    int mode = 1;               // 0 never tune, 1 tune unknown keys, 2 tune every key once more
    std::string file;
    bool env_read = false;
};
TuneState &tune_state()
{
    static TuneState st;
    return st;
}

void tune_load_file_locked(TuneState &st, const std::string &path)
{
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return;
    TuneKey k{};
    int v = 0;
    while (std::fscanf(f, "%d %d %d %d %d %d %d %d", &k.kind, &k.k, &k.bits, &k.h, &k.logn, &k.logdeg, &k.loghub,
                       &v) == 8)
        st.choice[k] = v;
    std::fclose(f);
}

void tune_env_locked(TuneState &st)
{
    if (st.env_read) return;
    st.env_read = true;
    const char *p = std::getenv("MC_AUTOTUNE_CACHE");
    if (p && *p) {
        st.file = p;
        tune_load_file_locked(st, st.file);
    }
}

int ilog2(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }
}  // namespace

static TuneKey tune_key(int kind, int k, int count_bits, int h, int64_t n, int64_t nnz, int64_t max_degree)
{
    const double nn = (double)std::max<int64_t>(n, 1);
    return TuneKey{kind, k, count_bits, h, ilog2((double)n), ilog2((double)nnz * (double)nnz / (nn * nn)),
                   ilog2((double)max_degree + 1)};
}

// Run `launch(candidate)` for the tuned candidate of `key`; when tuning is
// allowed and the key is new (or mode 2), time every candidate first.
template <typename F>
static void run_tuned(TuneKey key, int ncand, bool allow, cudaStream_t s, F &&launch)
{
    TuneState &st = tune_state();
    int v = -1;
    bool tune = false;
    {
        std::lock_guard<std::mutex> lock(st.mu);
        tune_env_locked(st);
        auto it = st.choice.find(key);
        if (it != st.choice.end()) v = it->second;
        tune = allow && st.mode > 0 && (v < 0 || (st.mode == 2 && !st.retuned.count(key)));
    }
    if (tune) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        MC_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) tune = false;
    }
    if (tune) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        MC_CUDA(cudaEventCreate(&e0));
        MC_CUDA(cudaEventCreate(&e1));
        // three rounds over the candidates, each candidate's best time
        // counts: every candidate meets the caches as the others left them
        float best[8];
        bool ok[8];
        for (int c = 0; c < ncand && c < 8; ++c) { best[c] = 0.f; ok[c] = true; }
        for (int rep = 0; rep < 3; ++rep)
            for (int c = 0; c < ncand && c < 8; ++c) {
                if (!ok[c]) continue;
                MC_CUDA(cudaEventRecord(e0, s));
                if (!launch(c)) { ok[c] = false; continue; }
                MC_CUDA(cudaEventRecord(e1, s));
                MC_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                MC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rep == 0 || ms < best[c]) best[c] = ms;
            }
        int bv = -1;
        for (int c = 0; c < ncand && c < 8; ++c)
            if (ok[c] && (bv < 0 || best[c] < best[bv])) bv = c;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        v = bv < 0 ? 0 : bv;
        std::lock_guard<std::mutex> lock(st.mu);
        st.choice[key] = v;
        st.retuned.insert(key);
        if (!st.file.empty()) {
            if (FILE *f = std::fopen(st.file.c_str(), "a")) {
                std::fprintf(f, "%d %d %d %d %d %d %d %d\n", key.kind, key.k, key.bits, key.h, key.logn, key.logdeg,
                             key.loghub, v);
                std::fclose(f);
            }
        }
    }
    if (v < 0 || !launch(v)) launch(0);
}

template <typename CT> static void build_levels(mc_tables *t, int *err, cudaStream_t s, bool allow_tune)
{
    const mc_graph *g = t->g;
    const Geometry &G = t->geo;
    const int k = t->k;
    const int64_t n = g->n;
    if (n == 0) return;
    // level 1 neighbour sums
    // colour blocks of every adjacency list, and the level-1 neighbour sums
    MC_LAUNCH("colour_blocks", s, colour_blocks_kernel<CT><<<grid_for(n, 256), 256, 0, s>>>(
                                      g->row_ptr, g->col, t->ecol, t->colors, n, k, t->scol, t->coff,
                                      (CT *)t->S[1]));
    if (g->n_hubs) {
        uint32_t *ccnt = t->ccnt;
        MC_LAUNCH("colour_blocks_hub", s, hub_chunk_counts_kernel<<<grid_for(g->n_chunks * 32, 256), 256, 0, s>>>(
                                              t->ecol, g->chunk_e0, g->chunk_e1, g->n_chunks, k, ccnt));
        MC_LAUNCH("colour_blocks_hub", s, hub_chunk_prefix_kernel<CT><<<grid_for(g->n_hubs * 32, 256), 256, 0, s>>>(
                                              t->colors, g->hub_node, g->hub_chunk0, g->n_hubs, k, ccnt, t->coff,
                                              (CT *)t->S[1]));
        MC_LAUNCH("colour_blocks_hub", s, hub_chunk_scatter_kernel<<<grid_for(g->n_chunks * 32, 256), 256, 0, s>>>(
                                              g->col, t->ecol, g->row_ptr, g->chunk_node, g->chunk_e0, g->chunk_e1,
                                              g->n_chunks, k, ccnt, t->coff, t->scol));
    }
    MergeArgs ma{};
    for (int h = 1; h <= k; ++h) {
        ma.c[h] = t->c[h];
        ma.S[h] = t->S[h];
        ma.Wc[h] = G.Wc[h];
        ma.Ws[h] = G.Ws[h];
        if (h <= MAXK) ma.div[h] = make_div(h);
    }
    ma.n = n;
    ma.err = err;
    for (int h = 2; h <= k; ++h) {
        if (t->skip_round && h == k - 1) continue;  // round k-1 skipped: nothing reads it
        ma.info = t->m_info[h];
        ma.off = t->m_off[h];
        ma.terms = t->m_terms[h];
        ma.out = t->c[h];
        ma.W = G.Wc[h];
        ma.Bc = G.Bc[h];
        ma.R = shape_catalog().r[h];
        ma.program = &programs(k, t->skip_round).merge[h];
        ma.zero_root_colors = (t->zero_root && h == k) ? t->colors : nullptr;
        const TuneKey mkey = tune_key(1, k, (int)sizeof(CT) * 8, h, n, g->nnz, g->max_degree);
        run_tuned(mkey, MERGE_CANDIDATES, allow_tune, s, [&](int c) { return launch_merge<CT>(ma, h, c, s); });
        if (h <= k - 1) {
            GatherArgs ga{};
            ga.row_ptr = g->row_ptr;
            ga.col = g->col;
            ga.colors = t->colors;
            ga.ecol = t->ecol;
            ga.node_chunk0 = g->node_chunk0;
            ga.src = t->c[h];
            ga.dst = t->S[h];
            ga.partial = t->Sp[h];
            ga.chunk_node = g->chunk_node;
            ga.chunk_e0 = g->chunk_e0;
            ga.chunk_e1 = g->chunk_e1;
            ga.gmap = t->g_map[h];
            ga.n = n;
            ga.n_chunks = g->n_chunks;
            ga.k = k;
            ga.Bs = G.Bs[h];
            ga.Wc = G.Wc[h];
            ga.Ws = G.Ws[h];
            ga.err = err;
            ga.sched = g->sched;
            ga.n_small = g->n_small;
            const TuneKey gkey = tune_key(0, k, (int)sizeof(CT) * 8, h, n, g->nnz, g->max_degree);
            const int rh = shape_catalog().r[h];
            run_tuned(gkey, GATHER_CANDIDATES, allow_tune, s, [&](int c) { return launch_gather<CT>(ga, rh, h, c, s); });
            if (g->n_hubs) {
                MC_LAUNCH("hub_reduce", s, hub_reduce_small_kernel<CT><<<grid_for(g->n_hubs * G.Ws[h], 256), 256, 0, s>>>(
                    (CT *)t->Sp[h], (CT *)t->S[h], g->hub_node, g->hub_chunk0, g->n_hubs, G.Ws[h], err));
                if (g->n_big_hubs)
                    MC_LAUNCH("hub_reduce", s, hub_reduce_kernel<CT><<<grid_for(g->n_big_hubs * G.Ws[h] * 32, 256), 256, 0, s>>>(
                        (CT *)t->Sp[h], (CT *)t->S[h], g->hub_node, g->hub_chunk0, g->big_hub, g->n_big_hubs,
                        G.Ws[h], err));
            }
        }
    }
}

}  // namespace mc

using namespace mc;

// Every launch of a build for the colours in `colors`, on stream s, into the
// buffers of t: no allocation, no host read, no synchronisation (so a
// rebuild can be captured into a CUDA graph).
static void enqueue_build(mc_tables *t, const uint8_t *colors, cudaStream_t s, bool allow_tune)
{
    const mc_graph *g = t->g;
    const int64_t n = g->n;
    const int k = t->k;
    int *err = t->dev_err;
    MC_CUDA(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));
    if (n) {
        // the tables' own copy of the colours, checked before any kernel reads them
        if (colors != t->colors)
            MC_CUDA(cudaMemcpyAsync(t->colors, colors, (size_t)n, cudaMemcpyDefault, s));
        MC_LAUNCH("check_colours", s, check_colours_kernel<<<grid_for(n, 256), 256, 0, s>>>(t->colors, n, k, err));
    }
    if (g->nnz)
        MC_LAUNCH("edge_colours", s, edge_colours_kernel<<<grid_for(g->nnz, 256), 256, 0, s>>>(
                                         g->col, t->colors, g->nnz, t->ecol));
    if (t->bits == 64) build_levels<uint64_t>(t, err, s, allow_tune);
    else build_levels<u128>(t, err, s, allow_tune);
    // root index of the top level (the level sampled by default); the other
    // levels get theirs on first use
    if (n) {
        launch_row_totals(t, k, ~0ull, ~0ull, t->prefix[k], err, s);
        inclusive_scan_u128_buf(t->prefix[k], n, err, t->scan_tmp, s);
        build_buckets(t->prefix[k], n, t->nbucket, t->dev_D, t->bucket[k], s);
    }
}

// Read the level-k total, the bucket width and the error flags back.
static void finish_build(mc_tables *t, cudaStream_t s)
{
    const int64_t n = t->g->n;
    int herr = 0;
    u128 R = 0, D = 1;
    MC_CUDA(cudaMemcpyAsync(&herr, t->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (n) {
        MC_CUDA(cudaMemcpyAsync(&R, t->prefix[t->k] + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(&D, t->dev_D, sizeof(u128), cudaMemcpyDeviceToHost, s));
    }
    MC_CUDA(cudaStreamSynchronize(s));
    if (herr & ERR_COLOUR) throw Error(MC_E_INVALID, "a colour is >= k");
    if (herr & ERR_OVERFLOW)
        throw Error(MC_E_OVERFLOW, "a count does not fit in " + std::to_string(t->bits) + " bits");
    if (herr & ERR_INEXACT) throw Error(MC_E_INTERNAL, "a merge numerator is not divisible by beta");
    t->R[t->k] = R;
    t->bucketD[t->k] = D;
}

extern "C" mc_status mc_build_tables(const mc_graph *g, const uint8_t *colors, int k, int count_bits,
                                     uint32_t flags, const mc_allocator *alloc, void *stream,
                                     mc_tables **out)
{
    if (out) *out = nullptr;
    mc_tables *t = nullptr;
    mc_status st = guarded([&] {
        MC_REQUIRE(out && g, "graph or out is NULL");
        MC_REQUIRE(colors || g->n == 0, "colors is NULL");
        if (k < 2 || k > MAXK) throw Error(MC_E_UNSUPPORTED, "k must be in 2..8");
        MC_REQUIRE(count_bits == 64 || count_bits == 128, "count_bits must be 64 or 128");
        MC_REQUIRE((flags & ~(MC_BUILD_ZERO_ROOT | MC_BUILD_SKIP_ROUND | MC_BUILD_SUCCINCT | MC_BUILD_VARLEN)) == 0,
                   "unknown flags");
        if (flags & MC_BUILD_SKIP_ROUND) {
            MC_REQUIRE(k >= 4, "round skipping needs k >= 4");
            MC_REQUIRE(!(flags & MC_BUILD_ZERO_ROOT), "round skipping and zero-rooting do not combine");
        }
        cudaStream_t s = (cudaStream_t)stream;
        t = new mc_tables();
        t->g = g;
        t->k = k;
        t->bits = count_bits;
        t->zero_root = flags & MC_BUILD_ZERO_ROOT;
        t->skip_round = flags & MC_BUILD_SKIP_ROUND;
        t->varlen = flags & MC_BUILD_VARLEN;
        const bool pack = (flags & (MC_BUILD_SUCCINCT | MC_BUILD_VARLEN)) != 0;
        t->geo = make_geometry(k);
        t->arena.stream = s;
        if (alloc) { t->arena.alloc.a = *alloc; t->arena.alloc.custom = true; }
        const int64_t n = g->n;
        const Geometry &G = t->geo;
        const size_t cb = count_bits / 8;
        // every buffer a build writes, kept for rebuilds
        t->dev_err = t->arena.get<int>(4);
        t->dev_D = t->arena.get<u128>(1);
        t->scan_tmp = t->arena.get<u128>((size_t)std::max<int64_t>(scan_tiles(n), 1));
        if (g->n_hubs) t->ccnt = t->arena.get<uint32_t>((size_t)g->n_chunks * k);
        t->colors = t->arena.get<uint8_t>((size_t)n);
        t->ecol = t->arena.get<uint8_t>((size_t)g->nnz);
        t->scol = t->arena.get<uint32_t>((size_t)g->nnz);
        t->coff = t->arena.get<int32_t>((size_t)n * (k + 1));
        // programs
        const Programs &P = programs(k, t->skip_round);
        for (int j = 0; j < 32; ++j) t->copies_k[j] = P.copies[j];
        for (int h = 2; h <= k; ++h) {
            if (t->level_missing(h)) continue;
            const MergeLevel &M = P.merge[h];
            t->m_info[h] = t->arena.get<int32_t>(M.info.size());
            t->m_off[h] = t->arena.get<int32_t>(M.offset.size());
            t->m_terms[h] = t->arena.get<uint32_t>(M.terms.size());
            MC_CUDA(cudaMemcpyAsync(t->m_info[h], M.info.data(), M.info.size() * 4, cudaMemcpyHostToDevice, s));
            MC_CUDA(cudaMemcpyAsync(t->m_off[h], M.offset.data(), M.offset.size() * 4, cudaMemcpyHostToDevice, s));
            MC_CUDA(cudaMemcpyAsync(t->m_terms[h], M.terms.data(), M.terms.size() * 4, cudaMemcpyHostToDevice, s));
        }
        for (int h = 1; h <= k - 1; ++h) {
            if (t->level_missing(h)) continue;
            const GatherLevel &L = P.gather[h];
            t->g_map[h] = t->arena.get<int16_t>(L.map.size());
            MC_CUDA(cudaMemcpyAsync(t->g_map[h], L.map.data(), L.map.size() * 2, cudaMemcpyHostToDevice, s));
        }
        // tables
        for (int h = 2; h <= k; ++h)
            if (!t->level_missing(h)) t->c[h] = t->arena.get<uint8_t>((size_t)n * G.Wc[h] * cb);
        for (int h = 1; h <= k - 1; ++h)
            if (!t->level_missing(h)) t->S[h] = t->arena.get<uint8_t>((size_t)n * G.Ws[h] * cb);
        for (int h = 2; h <= k - 1; ++h)
            if (!t->level_missing(h)) t->Sp[h] = t->arena.get<uint8_t>((size_t)g->n_chunks * G.Ws[h] * cb);
        t->nbucket = bucket_count(n);
        t->prefix[k] = t->arena.get<u128>((size_t)n);
        t->bucket[k] = t->arena.get<uint32_t>((size_t)t->nbucket + 1);
        enqueue_build(t, colors, s, true);
        finish_build(t, s);
        if (pack) {
            pack_tables(t, s);
            t->packed = true;
        }
    });
    if (st != MC_OK) { delete t; return st; }
    *out = t;
    return MC_OK;
}

extern "C" mc_status mc_rebuild_tables(mc_tables *t, const uint8_t *colors, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t, "tables is NULL");
        MC_REQUIRE(colors || t->g->n == 0, "colors is NULL");
        if (t->packed) throw Error(MC_E_UNSUPPORTED, "packed (succinct) tables cannot be rebuilt in place");
        std::lock_guard<std::mutex> lock(t->idx_mu);
        enqueue_build(t, colors, (cudaStream_t)stream, false);
        t->stale = true;
        t->broken.clear();
        for (int h = 2; h < t->k; ++h) t->level_stale[h] = t->prefix[h] != nullptr;
    });
}

void mc::refresh_tables(const mc_tables *tc, cudaStream_t s, bool force)
{
    mc_tables *t = const_cast<mc_tables *>(tc);
    std::lock_guard<std::mutex> lock(t->idx_mu);
    if (force) {
        // a replayed capture runs no host code: treat the device state as new
        t->stale = true;
        t->broken.clear();
        for (int h = 2; h < t->k; ++h) t->level_stale[h] = t->prefix[h] != nullptr;
    }
    if (!t->broken.empty()) throw Error(MC_E_INVALID, "the last rebuild failed: " + t->broken);
    if (!t->stale) return;
    try {
        finish_build(t, s);
    } catch (const Error &e) {
        t->broken = e.what();
        throw;
    }
    t->stale = false;
}

extern "C" mc_status mc_tables_status(const mc_tables *t, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t, "tables is NULL");
        refresh_tables(t, (cudaStream_t)stream, true);
    });
}

void mc::ensure_level_index(const mc_tables *tc, int h, cudaStream_t s)
{
    mc_tables *t = const_cast<mc_tables *>(tc);
    refresh_tables(t, s);
    std::lock_guard<std::mutex> lock(t->idx_mu);
    if (h < 2 || (t->prefix[h] && !t->level_stale[h])) return;
    if (t->level_missing(h)) throw Error(MC_E_INVALID, "level h was skipped (round skipping)");
    const int64_t n = t->g->n;
    Arena scratch(true);
    scratch.alloc = t->arena.alloc;
    scratch.stream = s;
    int *err = scratch.get<int>(1);
    u128 *dD = scratch.get<u128>(1);
    MC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    // a stale index (from an older colouring) is rebuilt in its own buffers
    u128 *p = t->prefix[h] ? t->prefix[h] : t->arena.get<u128>((size_t)n);
    uint32_t *bk = t->bucket[h] ? t->bucket[h] : t->arena.get<uint32_t>((size_t)t->nbucket + 1);
    launch_row_totals(t, h, ~0ull, ~0ull, p, err, s);
    inclusive_scan_u128(p, n, err, scratch, s);
    build_buckets(p, n, t->nbucket, dD, bk, s);
    u128 R = 0, D = 1;
    int herr = 0;
    if (n) {
        MC_CUDA(cudaMemcpyAsync(&R, p + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(&D, dD, sizeof(u128), cudaMemcpyDeviceToHost, s));
    }
    MC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error(MC_E_OVERFLOW, "a level total does not fit in 128 bits");
    t->R[h] = R;
    t->bucketD[h] = D;
    t->bucket[h] = bk;
    t->prefix[h] = p;  // published last
    t->level_stale[h] = false;
}

extern "C" void mc_free_tables(mc_tables *t)
{
    if (!t) return;
    mc_graph *owned = t->owned_graph;
    delete t;
    mc_free_graph(owned);
}

// Rooted total R of level h over the nodes [lo, hi): all shapes (j < 0,
// from the cached root index) or the rootings of unrooted shape j.
static u128 level_rooted_total(const mc_tables *t, int h, int j, int64_t lo, int64_t hi, cudaStream_t s)
{
    const ShapeCatalog &cat = shape_catalog();
    const int64_t n = t->g->n;
    if (h == 1) return j > 0 ? 0 : (u128)(hi - lo);
    if (hi <= lo) return 0;
    // the level's node prefix, read at the range's ends
    const u128 *pre = nullptr;
    Arena scratch(true);
    scratch.alloc = t->arena.alloc;
    scratch.stream = s;
    int *err = scratch.get<int>(1);
    MC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (j < 0) {
        ensure_level_index(t, h, s);
        pre = t->prefix[h];
    } else {
        uint64_t a0 = 0, a1 = 0;
        for (int i = 0; i < cat.r[h]; ++i)
            if (cat.shapes[cat.gid(h, i)].unrooted == j) {
                if (i < 64) a0 |= 1ull << i; else a1 |= 1ull << (i - 64);
            }
        u128 *tot = scratch.get<u128>((size_t)n);
        launch_row_totals(t, h, a0, a1, tot, err, s);
        inclusive_scan_u128(tot, n, err, scratch, s);
        pre = tot;
    }
    u128 top = 0, base = 0;
    int herr = 0;
    MC_CUDA(cudaMemcpyAsync(&top, pre + (hi - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
    if (lo > 0) MC_CUDA(cudaMemcpyAsync(&base, pre + (lo - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error(MC_E_OVERFLOW, "level total does not fit in 128 bits");
    return top - base;
}

// Copies of unrooted shape j from its rooted total: R / h (one rooted copy
// per node), R at a zero-rooted level k, R / a_j at a round-skipped level k
// (a_j = 0: the star, not counted).
u128 mc::unrooted_from_rooted(const mc_tables *t, int h, int j, u128 R)
{
    u128 div = (u128)t->copies_div(h);
    if (t->skip_round && h == t->k) {
        div = (u128)t->copies_k[j];
        if (div == 0) {
            if (R != 0) throw Error(MC_E_INTERNAL, "an uncounted shape has counts");
            return 0;
        }
    }
    if (R % div != 0) throw Error(MC_E_INTERNAL, "rooted total not divisible by h");
    return R / div;
}

extern "C" mc_status mc_total_range(const mc_tables *t, int h, int32_t unrooted_shape, int64_t node_lo,
                                    int64_t node_hi, uint64_t rooted[2], uint64_t unrooted_count[2], void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t && rooted && unrooted_count, "NULL argument");
        refresh_tables(t, (cudaStream_t)stream);
        MC_REQUIRE(h >= 1 && h <= t->k, "h must be in 1..k");
        MC_REQUIRE(!t->level_missing(h), "level h was skipped (round skipping)");
        const ShapeCatalog &cat = shape_catalog();
        MC_REQUIRE(unrooted_shape >= -1 && unrooted_shape < cat.n_unrooted[h], "unrooted shape out of range");
        const int64_t n = t->g->n;
        int64_t lo = node_lo, hi = node_hi;
        if (hi <= 0 && lo <= 0) { lo = 0; hi = n; }
        if (hi <= 0) hi = n;
        MC_REQUIRE(lo >= 0 && lo <= hi && hi <= n, "node range out of bounds");
        cudaStream_t s = (cudaStream_t)stream;
        const u128 R = level_rooted_total(t, h, unrooted_shape, lo, hi, s);
        u128 U = 0;
        if (unrooted_shape >= 0) {
            U = unrooted_from_rooted(t, h, unrooted_shape, R);
        } else if (t->skip_round && h == t->k) {
            // per-shape divisors differ: t = sum_j R_j / a_j
            for (int j = 0; j < cat.n_unrooted[h]; ++j)
                U += unrooted_from_rooted(t, h, j, level_rooted_total(t, h, j, lo, hi, s));
        } else {
            const u128 div = (u128)t->copies_div(h);
            if (R % div != 0) throw Error(MC_E_INTERNAL, "rooted total not divisible by h");
            U = R / div;
        }
        rooted[0] = (uint64_t)R;
        rooted[1] = (uint64_t)(R >> 64);
        unrooted_count[0] = (uint64_t)U;
        unrooted_count[1] = (uint64_t)(U >> 64);
    });
}

extern "C" mc_status mc_total(const mc_tables *t, int h, int32_t unrooted_shape, uint64_t rooted[2],
                              uint64_t unrooted_count[2], void *stream)
{
    return mc_total_range(t, h, unrooted_shape, 0, 0, rooted, unrooted_count, stream);
}

// ---------------------------------------------------------------------------
// batches: several (graph, colouring) instances side by side as one disjoint
// union, built in one pass (one launch per kernel for the whole batch)
// ---------------------------------------------------------------------------
__global__ void concat_csr_kernel(const int64_t *__restrict__ rp, const uint32_t *__restrict__ col, int64_t n,
                                  int64_t nnz, int64_t noff, int64_t eoff, int64_t *__restrict__ urp,
                                  uint32_t *__restrict__ ucol)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz || i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) urp[noff + i] = eoff + rp[i];
        if (i < nnz) ucol[eoff + i] = col[i] + (uint32_t)noff;
    }
}

extern "C" mc_status mc_build_tables_batch(int count, const mc_graph *const *graphs, const uint8_t *const *colors,
                                           int k, int count_bits, uint32_t flags, const mc_allocator *alloc,
                                           void *stream, mc_tables **out, int64_t *node_offsets)
{
    if (out) *out = nullptr;
    mc_graph *ug = nullptr;
    mc_tables *t = nullptr;
    mc_status st = guarded([&] {
        MC_REQUIRE(out && node_offsets && graphs && colors && count >= 1, "bad batch arguments");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<int64_t> noff(count + 1, 0), eoff(count + 1, 0);
        for (int i = 0; i < count; ++i) {
            MC_REQUIRE(graphs[i] && (colors[i] || graphs[i]->n == 0), "NULL graph or colours in batch");
            noff[i + 1] = noff[i] + graphs[i]->n;
            eoff[i + 1] = eoff[i] + graphs[i]->nnz;
        }
        const int64_t N = noff[count], NNZ = eoff[count];
        MC_REQUIRE(N < (int64_t)0xffffffffLL, "batch has too many nodes");
        Arena scratch(true);
        if (alloc) { scratch.alloc.a = *alloc; scratch.alloc.custom = true; }
        scratch.stream = s;
        int64_t *urp = scratch.get<int64_t>((size_t)N + 1);
        uint32_t *ucol = scratch.get<uint32_t>((size_t)(NNZ > 0 ? NNZ : 1));
        uint8_t *ucolors = scratch.get<uint8_t>((size_t)(N > 0 ? N : 1));
        for (int i = 0; i < count; ++i) {
            const mc_graph *g = graphs[i];
            if (g->n == 0) continue;
            MC_LAUNCH("concat_csr", s, concat_csr_kernel<<<grid_for(std::max(g->n, g->nnz), 256), 256, 0, s>>>(
                                           g->row_ptr, g->col, g->n, g->nnz, noff[i], eoff[i], urp, ucol));
            MC_CUDA(cudaMemcpyAsync(ucolors + noff[i], colors[i], (size_t)g->n, cudaMemcpyDefault, s));
        }
        MC_CUDA(cudaMemcpyAsync(urp + N, &NNZ, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        mc_status s2 = mc_load_graph(N, NNZ, urp, ucol, MC_GRAPH_DEVICE_PTRS | MC_GRAPH_TRUSTED, alloc, stream, &ug);
        if (s2 != MC_OK) throw Error(s2, std::string("batch graph: ") + mc_last_error());
        s2 = mc_build_tables(ug, ucolors, k, count_bits, flags, alloc, stream, &t);
        if (s2 != MC_OK) throw Error(s2, std::string("batch build: ") + mc_last_error());
        t->owned_graph = ug;
        ug = nullptr;
        for (int i = 0; i <= count; ++i) node_offsets[i] = noff[i];
    });
    if (st != MC_OK) {
        delete t;
        mc_free_graph(ug);
        return st;
    }
    *out = t;
    return MC_OK;
}

// number of non-zero entries among n words (or pairs of words for u128)
template <typename CT>
__global__ void nonzeros_kernel(const CT *__restrict__ x, int64_t n, unsigned long long *count)
{
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += x[i] != 0;
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

extern "C" mc_status mc_table_nonzeros(const mc_tables *t, int h, int which, int64_t *count, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t && count, "NULL argument");
        refresh_tables(t, (cudaStream_t)stream);
        MC_REQUIRE(which == 0 || which == 1, "which must be 0 (c) or 1 (S)");
        MC_REQUIRE(h >= 1 && h <= (which ? t->k - 1 : t->k), "h out of range");
        MC_REQUIRE(!t->level_missing(h), "level h was skipped (round skipping)");
        const int64_t n = t->g->n;
        if (which == 0 && h == 1) { *count = n; return; }
        const int64_t m = n * (which ? t->geo.Ws[h] : t->geo.Wc[h]);
        cudaStream_t s = (cudaStream_t)stream;
        if (t->packed) {  // the packed level holds exactly its non-zero entries
            int64_t c = 0;
            if (n) {
                MC_CUDA(cudaMemcpyAsync(&c, (which ? t->ps : t->pc)[h].off + n, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, s));
                MC_CUDA(cudaStreamSynchronize(s));
            }
            *count = c;
            return;
        }
        Arena scratch(true);
        scratch.alloc = t->arena.alloc;
        scratch.stream = s;
        unsigned long long *d = scratch.get<unsigned long long>(1), hc = 0;
        MC_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), s));
        const void *src = which ? t->S[h] : t->c[h];
        if (m > 0) {
            if (t->bits == 64)
                MC_LAUNCH("nonzeros", s, nonzeros_kernel<uint64_t><<<grid_for(m, 256), 256, 0, s>>>((const uint64_t *)src, m, d));
            else
                MC_LAUNCH("nonzeros", s, nonzeros_kernel<u128><<<grid_for(m, 256), 256, 0, s>>>((const u128 *)src, m, d));
        }
        MC_CUDA(cudaMemcpyAsync(&hc, d, sizeof(hc), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        *count = (int64_t)hc;
    });
}

extern "C" mc_status mc_table_layout(const mc_tables *t, int h, int which, int64_t *row_entries,
                                     int *entry_bytes)
{
    return guarded([&] {
        MC_REQUIRE(t, "tables is NULL");
        MC_REQUIRE(which == 0 || which == 1, "which must be 0 (c) or 1 (S)");
        MC_REQUIRE(h >= 1 && h <= (which ? t->k - 1 : t->k), "h out of range");
        MC_REQUIRE(!t->level_missing(h), "level h was skipped (round skipping)");
        if (row_entries) *row_entries = which ? t->geo.Ws[h] : t->geo.Wc[h];
        if (entry_bytes) *entry_bytes = t->bits / 8;
    });
}

extern "C" mc_status mc_read_table(const mc_tables *t, int h, int which, void *dst, size_t dst_bytes,
                                   int dst_on_device, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t && dst, "NULL argument");
        refresh_tables(t, (cudaStream_t)stream);
        MC_REQUIRE(which == 0 || which == 1, "which must be 0 (c) or 1 (S)");
        MC_REQUIRE(h >= 1 && h <= (which ? t->k - 1 : t->k), "h out of range");
        MC_REQUIRE(!t->level_missing(h), "level h was skipped (round skipping)");
        const int64_t W = which ? t->geo.Ws[h] : t->geo.Wc[h];
        const size_t bytes = (size_t)t->g->n * W * (t->bits / 8);
        MC_REQUIRE(dst_bytes >= bytes, "dst too small");
        cudaStream_t s = (cudaStream_t)stream;
        if (bytes == 0) return;
        if (which == 0 && h == 1) {
            if (dst_on_device) {
                MC_LAUNCH("fill_ones", s, fill_ones_kernel<<<grid_for(t->g->n, 256), 256, 0, s>>>(dst, t->g->n, t->bits / 8));
            } else {
                std::memset(dst, 0, bytes);
                for (int64_t v = 0; v < t->g->n; ++v) ((uint8_t *)dst)[v * (t->bits / 8)] = 1;
            }
        } else if (t->packed) {
            if (dst_on_device) {
                launch_unpack(t, h, which, dst, s);
            } else {
                Arena scratch(true);
                scratch.alloc = t->arena.alloc;
                scratch.stream = s;
                void *tmp = scratch.get<uint8_t>(bytes);
                launch_unpack(t, h, which, tmp, s);
                MC_CUDA(cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, s));
                MC_CUDA(cudaStreamSynchronize(s));
            }
        } else {
            const void *src = which ? t->S[h] : t->c[h];
            MC_CUDA(cudaMemcpyAsync(dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        }
        MC_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" mc_status mc_autotune(int mode, const char *cache_file)
{
    return guarded([&] {
        MC_REQUIRE(mode >= 0 && mode <= 2, "mode must be 0, 1 or 2");
        TuneState &st = tune_state();
        std::lock_guard<std::mutex> lock(st.mu);
        tune_env_locked(st);
        st.mode = mode;
        if (mode == 2) st.retuned.clear();
        if (cache_file) {  // "" stops appending
            st.file = cache_file;
            if (!st.file.empty()) tune_load_file_locked(st, st.file);
        }
    });
}

extern "C" int mc_autotune_choice(int kind, int k, int count_bits, int h, int64_t n, int64_t nnz, int64_t max_degree)
{
    const TuneKey key = tune_key(kind, k, count_bits, h, n, nnz, max_degree);
    TuneState &st = tune_state();
    std::lock_guard<std::mutex> lock(st.mu);
    tune_env_locked(st);
    auto it = st.choice.find(key);
    return it == st.choice.end() ? -1 : it->second;
}

extern "C" mc_status mc_autotune_set(int kind, int k, int count_bits, int h, int64_t n, int64_t nnz,
                                     int64_t max_degree, int choice)
{
    return guarded([&] {
        MC_REQUIRE(kind == 0 || kind == 1, "kind must be 0 (neighbour sums) or 1 (merge)");
        MC_REQUIRE(choice >= 0 && choice < (kind == 0 ? GATHER_CANDIDATES : MERGE_CANDIDATES), "no such schedule");
        const TuneKey key = tune_key(kind, k, count_bits, h, n, nnz, max_degree);
        TuneState &st = tune_state();
        std::lock_guard<std::mutex> lock(st.mu);
        tune_env_locked(st);
        st.choice[key] = choice;
    });
}
