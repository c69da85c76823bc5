// sample.cu -- graphlet classes (Section 4.4.3), uniform and shape-restricted
// colourful treelet sampling (Section 2.2; sample(T) of Section 4.1), the
// uniform estimator (Section 2.2) and adaptive graphlet sampling (Algorithm
// AGS, Section 4.1).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "internal.h"

namespace mc {

void inclusive_scan_u128(u128 *x, int64_t n, int *err, Arena &scratch, cudaStream_t s);

enum : int { SERR_SEARCH = 1, SERR_CLASS = 2 };

// ---------------------------------------------------------------------------
// Graphlet classes.  Adjacency word of a labelled h-node graph: the pairs
// (i, j), i < j, in lexicographic order, the first pair in the most
// significant of the P = C(h,2) bits.  Canonical word: the minimum over all
// relabelings.  The connected classes of size h are found from those of size
// h-1 (every connected graph has a node whose removal leaves it connected):
// each (h-1)-class plus a new node joined to a non-empty node set is
// canonicalised on the GPU (all h! relabelings per candidate), and the
// distinct results, ascending, are the class codes.  The lookup table maps
// every word of a connected graph to its class: one GPU thread per (class,
// relabeling) writes the relabeled word's entry.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int pair_pos(int h, int i, int j)
{
    const int P = h * (h - 1) / 2;
    return P - 1 - (i * (2 * h - i - 1) / 2 + (j - i - 1));
}

__device__ __forceinline__ uint32_t relabel_word(uint32_t w, int h, const int *p)
{
    // new labels i < j are adjacent when old labels p[i], p[j] are
    uint32_t out = 0;
    for (int i = 0; i < h; ++i)
        for (int j = i + 1; j < h; ++j) {
            const int a = min(p[i], p[j]), b = max(p[i], p[j]);
            if ((w >> pair_pos(h, a, b)) & 1u) out |= 1u << pair_pos(h, i, j);
        }
    return out;
}

__global__ void canon_kernel(const uint32_t *cand, int64_t nc, int h, uint32_t *out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = cand[t];
        int p[MAXK], c[MAXK];
        for (int i = 0; i < h; ++i) { p[i] = i; c[i] = 0; }
        uint32_t best = relabel_word(w, h, p);
        int i = 1;
        while (i < h) {  // Heap's algorithm: every permutation once
            if (c[i] < i) {
                const int a = (i & 1) ? c[i] : 0;
                const int tmp = p[a]; p[a] = p[i]; p[i] = tmp;
                const uint32_t x = relabel_word(w, h, p);
                if (x < best) best = x;
                ++c[i];
                i = 1;
            } else {
                c[i] = 0;
                ++i;
            }
        }
        out[t] = best;
    }
}

__global__ void fill_lut_kernel(const uint32_t *codes, int ncls, int h, int64_t nperm, uint16_t *lut)
{
    const int64_t total = (int64_t)ncls * nperm;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int cls = (int)(t / nperm);
        int64_t r = t - (int64_t)cls * nperm;
        // permutation number r in the factorial number system
        int p[MAXK], used = 0;
        int64_t f = nperm;
        for (int i = 0; i < h; ++i) {
            f /= (h - i);
            int d = (int)(r / f);
            r -= d * f;
            int x = 0;
            for (;; ++x)
                if (!((used >> x) & 1) && d-- == 0) break;
            used |= 1 << x;
            p[i] = x;
        }
        lut[relabel_word(codes[cls], h, p)] = (uint16_t)cls;
    }
}

struct ClassCatalog {
    int h = 0;
    std::vector<uint32_t> codes;
    uint16_t *lut = nullptr;  // device, 2^C(h,2) entries (0xffff: not connected)
    bool sigma_ready = false;
    std::vector<int64_t> sigma_i, sigma_ij;
};

static std::mutex g_cls_mutex;
static std::map<std::pair<int, int>, ClassCatalog *> g_cls;

static int64_t factorial(int h)
{
    int64_t f = 1;
    for (int i = 2; i <= h; ++i) f *= i;
    return f;
}

static ClassCatalog *class_catalog_locked(int h);

static ClassCatalog *build_classes(int h)
{
    ClassCatalog *cc = new ClassCatalog();
    cc->h = h;
    const int P = h * (h - 1) / 2;
    if (h == 1) {
        cc->codes = {0u};
    } else {
        const ClassCatalog *prev = class_catalog_locked(h - 1);
        std::vector<uint32_t> cand;
        for (uint32_t R : prev->codes)
            for (unsigned S = 1; S < (1u << (h - 1)); ++S) {
                uint32_t w = 0;
                for (int i = 0; i < h - 1; ++i)
                    for (int j = i + 1; j < h - 1; ++j)
                        if ((R >> pair_pos(h - 1, i, j)) & 1u) w |= 1u << pair_pos(h, i, j);
                for (int i = 0; i < h - 1; ++i)
                    if ((S >> i) & 1u) w |= 1u << pair_pos(h, i, h - 1);
                cand.push_back(w);
            }
        uint32_t *dc = nullptr, *dout = nullptr;
        MC_CUDA(cudaMalloc(&dc, cand.size() * 4));
        MC_CUDA(cudaMalloc(&dout, cand.size() * 4));
        MC_CUDA(cudaMemcpy(dc, cand.data(), cand.size() * 4, cudaMemcpyHostToDevice));
        MC_LAUNCH("canon", nullptr, canon_kernel<<<grid_for((int64_t)cand.size(), 128), 128>>>(dc, (int64_t)cand.size(), h, dout));
        std::vector<uint32_t> canon(cand.size());
        MC_CUDA(cudaMemcpy(canon.data(), dout, cand.size() * 4, cudaMemcpyDeviceToHost));
        cudaFree(dc);
        cudaFree(dout);
        std::sort(canon.begin(), canon.end());
        canon.erase(std::unique(canon.begin(), canon.end()), canon.end());
        cc->codes = canon;
    }
    if (cc->codes.size() > 0xffff) throw Error(MC_E_INTERNAL, "too many classes");
    const size_t nw = (size_t)1 << P;
    MC_CUDA(cudaMalloc(&cc->lut, nw * sizeof(uint16_t)));
    MC_CUDA(cudaMemset(cc->lut, 0xff, nw * sizeof(uint16_t)));
    uint32_t *dcodes = nullptr;
    MC_CUDA(cudaMalloc(&dcodes, cc->codes.size() * 4));
    MC_CUDA(cudaMemcpy(dcodes, cc->codes.data(), cc->codes.size() * 4, cudaMemcpyHostToDevice));
    const int64_t nperm = factorial(h);
    const int64_t total = (int64_t)cc->codes.size() * nperm;
    MC_LAUNCH("fill_lut", nullptr, fill_lut_kernel<<<grid_for(total, 256), 256>>>(dcodes, (int)cc->codes.size(), h, nperm, cc->lut));
    MC_CUDA(cudaDeviceSynchronize());
    cudaFree(dcodes);
    return cc;
}

static ClassCatalog *class_catalog_locked(int h)
{
    int dev = 0;
    MC_CUDA(cudaGetDevice(&dev));
    auto key = std::make_pair(dev, h);
    auto it = g_cls.find(key);
    if (it != g_cls.end()) return it->second;
    ClassCatalog *cc = build_classes(h);
    g_cls[key] = cc;
    return cc;
}

ClassCatalog *class_catalog(int h)
{
    if (h < 1 || h > MAXK) throw Error(MC_E_INVALID, "h must be in 1..8");
    std::lock_guard<std::mutex> lock(g_cls_mutex);
    return class_catalog_locked(h);
}

// sigma_ij by the paper's recipe (Section 4.4.3): build the tables of every
// class graph with each node its own colour; the colourful h-treelets are
// then exactly the spanning trees.  All classes go through one build, as a
// disjoint union.
__global__ void sigma_kernel(const uint64_t *c, int64_t n, int h, int W, const int8_t *unrooted_of,
                             int nu, unsigned long long *acc)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * W;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / W;
        const int s = (int)(t - v * W);  // one colour set (all colours) per shape
        const uint64_t x = c[t];
        if (x) atomicAdd(&acc[(v / h) * nu + unrooted_of[s]], (unsigned long long)x);
    }
}

static void ensure_sigma(ClassCatalog *cc)
{
    if (cc->sigma_ready) return;
    const int h = cc->h;
    const ShapeCatalog &cat = shape_catalog();
    const int nu = cat.n_unrooted[h];
    const int64_t ncls = (int64_t)cc->codes.size();
    cc->sigma_ij.assign((size_t)ncls * nu, 0);
    cc->sigma_i.assign((size_t)ncls, 0);
    if (h == 1) {
        cc->sigma_ij[0] = 1;
        cc->sigma_i[0] = 1;
        cc->sigma_ready = true;
        return;
    }
    // disjoint union: node i of class c is c * h + i, coloured i
    const int64_t n = ncls * h;
    std::vector<int64_t> rp((size_t)n + 1, 0);
    std::vector<uint32_t> col;
    std::vector<uint8_t> colors((size_t)n);
    for (int64_t c = 0; c < ncls; ++c)
        for (int i = 0; i < h; ++i) {
            const int64_t v = c * h + i;
            colors[v] = (uint8_t)i;
            for (int j = 0; j < h; ++j) {
                if (j == i) continue;
                const int a = std::min(i, j), b = std::max(i, j);
                if ((cc->codes[c] >> pair_pos(h, a, b)) & 1u) col.push_back((uint32_t)(c * h + j));
            }
            rp[v + 1] = (int64_t)col.size();
        }
    mc_graph *g = nullptr;
    mc_tables *t = nullptr;
    mc_status st = mc_load_graph(n, (int64_t)col.size(), rp.data(), col.data(), MC_GRAPH_TRUSTED, nullptr,
                                 nullptr, &g);
    if (st != MC_OK) throw Error(st, "sigma: load graph failed");
    uint8_t *dcol = nullptr;
    MC_CUDA(cudaMalloc(&dcol, (size_t)n));
    MC_CUDA(cudaMemcpy(dcol, colors.data(), (size_t)n, cudaMemcpyHostToDevice));
    st = mc_build_tables(g, dcol, h, 64, 0, nullptr, nullptr, &t);
    cudaFree(dcol);
    if (st != MC_OK) { mc_free_graph(g); throw Error(st, "sigma: build failed"); }
    std::vector<int8_t> uo(cat.r[h]);
    for (int s = 0; s < cat.r[h]; ++s) uo[s] = (int8_t)cat.shapes[cat.gid(h, s)].unrooted;
    int8_t *duo = nullptr;
    unsigned long long *dacc = nullptr;
    MC_CUDA(cudaMalloc(&duo, uo.size()));
    MC_CUDA(cudaMalloc(&dacc, (size_t)ncls * nu * 8));
    MC_CUDA(cudaMemcpy(duo, uo.data(), uo.size(), cudaMemcpyHostToDevice));
    MC_CUDA(cudaMemset(dacc, 0, (size_t)ncls * nu * 8));
    const int W = t->geo.Wc[h];  // = r_h: one colour set
    MC_LAUNCH("sigma", nullptr, sigma_kernel<<<grid_for(n * W, 256), 256>>>((const uint64_t *)t->c[h], n, h, W, duo, nu, dacc));
    std::vector<unsigned long long> acc((size_t)ncls * nu);
    MC_CUDA(cudaMemcpy(acc.data(), dacc, acc.size() * 8, cudaMemcpyDeviceToHost));
    cudaFree(duo);
    cudaFree(dacc);
    mc_free_tables(t);
    mc_free_graph(g);
    for (int64_t c = 0; c < ncls; ++c)
        for (int j = 0; j < nu; ++j) {
            const unsigned long long x = acc[(size_t)c * nu + j];
            if (x % (unsigned long long)h) throw Error(MC_E_INTERNAL, "sigma: rooted count not divisible by h");
            cc->sigma_ij[(size_t)c * nu + j] = (int64_t)(x / h);
            cc->sigma_i[(size_t)c] += (int64_t)(x / h);
        }
    cc->sigma_ready = true;
}

ClassCatalog *class_catalog_sigma(int h)
{
    ClassCatalog *cc = class_catalog(h);
    std::lock_guard<std::mutex> lock(g_cls_mutex);
    ensure_sigma(cc);
    return cc;
}

// ---------------------------------------------------------------------------
// Sampler: one warp per sample.
//   step 0  X = uniform(R); v = first node whose inclusive prefix exceeds X
//           (32-ary warp search); (T, C) = first entry of v's level-h row,
//           in (shape id, colour mask) order, whose running sum exceeds the
//           remainder (warp scan);
//   step s  for each decomposition node (T, C, x) in pre-order (T' before
//           T''): Y = uniform(beta_T c(T_C, x)); the block of colour sets
//           C'' (ascending mask) is found from the block weights
//           c(T'_{C\C''}, x) S(T'', C'', x); inside it, the neighbour u
//           (ascending) is the first whose running sum of c(T''_{C''}, u)
//           exceeds floor(Y' / c(T'_{C\C''}, x)) -- the same pair as a flat
//           scan over (C'', u) with weights c(T') c(T'').
// The h leaves of the decomposition are the sample's nodes; their induced
// subgraph is classified by the lookup table.
// ---------------------------------------------------------------------------
// Page-locked host memory (so device-to-host copies run asynchronously),
// one buffer per calling thread, grown on demand and kept for the thread's
// next calls: page-locking is slow, and a thread runs one call at a time.
static void *pinned_scratch(size_t bytes)
{
    struct Buf {
        void *p = nullptr;
        size_t n = 0;
        ~Buf() { if (p) cudaFreeHost(p); }
    };
    thread_local Buf b;
    if (b.n < bytes) {
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.n = 0;
        if (cudaMallocHost(&b.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            throw Error(MC_E_NOMEM, "page-locked host allocation failed");
        }
        b.n = bytes;
    }
    return b.p;
}

// A CUDA event, released with its scope.

struct EventHandle {
    cudaEvent_t e = nullptr;
    EventHandle() { MC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)); }
    ~EventHandle() { cudaEventDestroy(e); }
    EventHandle(const EventHandle &) = delete;
    EventHandle &operator=(const EventHandle &) = delete;
};

// One treelet's part of a launch that draws from several treelets: samples
// [end of the previous part, end) come from this root index, the first with
// sample index first_index.
struct SampleSeg {
    int64_t end;
    uint64_t first_index;
    const u128 *prefix;
    const uint32_t *bucket;
    u128 R, Xbase, D;
    uint64_t allow0, allow1;
};
static_assert(sizeof(SampleSeg) <= 128, "request admission charges 128 bytes per part");

struct SampleArgs {
    const int64_t *row_ptr;
    const uint32_t *col;
    const uint8_t *colors;
    const uint8_t *ecol;
    const uint32_t *scol;
    const int32_t *coff;
    int64_t n;
    const void *c[MAXK + 1];
    const void *S[MAXK + 1];
    PackedView pc[MAXK + 1], ps[MAXK + 1];  // the levels of packed (succinct) tables
    const void *Sp[MAXK + 1];   // per level: inclusive prefix of each hub's chunk sums
    const int32_t *node_chunk0; // first chunk of a hub, -1 for other nodes
    int Bc[MAXK + 1], Bs[MAXK + 1], Wc[MAXK + 1], Ws[MAXK + 1];
    int R_[MAXK + 1];           // rooted shapes per size: rows are set-major, entry (set, shape) at set * R_ + shape
    int k, h;
    const u128 *prefix;
    u128 R;                     // total of the node range sampled from
    u128 Xbase;                 // prefix before that range (0 for the whole graph)
    const uint32_t *bucket;     // root-search buckets (nb + 1 entries)
    u128 D;                     // bucket width
    uint64_t allow0, allow1;
    const SampleSeg *seg;       // nseg > 0: the launch's parts, each with its own root index and
    int nseg;                   // index stream (prefix .. allow1 above unused)
    int first[MAXK + 2];
    uint8_t sz[MAX_SHAPES], loc[MAX_SHAPES], lft[MAX_SHAPES], rgt[MAX_SHAPES], beta[MAX_SHAPES];
    uint8_t crank[1 << (MAXK - 1)];        // colex rank of a set of the k-1 relative colours
    uint8_t unrank[MAXK][36];              // i-th m-subset (ascending masks)
    uint8_t pi[28], pj[28];
    uint64_t seed, first_index;
    int64_t count;
    const uint16_t *lut;
    uint32_t *nodes, *roots;
    int32_t *shapes, *classes;
    unsigned long long *hist;
    unsigned long long *bytes;  // when set: data bytes read and written, counted item by item
    unsigned long long *next;   // when set: warps take batches of 32 samples from this counter
                                // (zero at launch) as they finish; else a fixed grid stride
    int ncls;
    int *err;
};

struct SampleSmem {
    uint8_t crank[1 << (MAXK - 1)];
    uint8_t unrank[MAXK][36];
};

// Entry idx of node x's level-h row of c or S: dense rows, or (PK) a binary
// search of the packed row's keys.
template <typename CT, bool PK>
__device__ __forceinline__ CT c_at(const SampleArgs &a, int h, int64_t x, int idx)
{
    if constexpr (PK) return (CT)packed_get(a.pc[h], x, idx);
    else return ((const CT *)a.c[h])[x * a.Wc[h] + idx];
}
template <typename CT, bool PK>
__device__ __forceinline__ CT s_at(const SampleArgs &a, int h, int64_t x, int idx)
{
    if constexpr (PK) return (CT)packed_get(a.ps[h], x, idx);
    else return ((const CT *)a.S[h])[x * a.Ws[h] + idx];
}

template <typename CT, typename V, bool PK>
__device__ __forceinline__ V count_at(const SampleArgs &a, const SampleSmem &sm, int g, unsigned C, uint32_t x, int cx)
{
    const int hg = a.sz[g];
    if (hg == 1) return 1;
    const unsigned rel = drop_colour(C & ~(1u << cx), cx);
    return (V)c_at<CT, PK>(a, hg, x, sm.crank[rel] * a.R_[hg] + a.loc[g]);
}

__device__ __forceinline__ uint64_t quotient(uint64_t a, uint64_t b) { return a / b; }
__device__ __forceinline__ u128 quotient(u128 a, u128 b)
{
    return ((a >> 64) == 0 && (b >> 64) == 0) ? (u128)((uint64_t)a / (uint64_t)b) : a / b;
}

// the set bits of `rest` selected by index mask `im` (i-th bit of im picks
// the i-th lowest set bit of rest)
__device__ __forceinline__ unsigned deposit(unsigned im, unsigned rest)
{
    unsigned out = 0;
    for (int i = 0; rest; ++i) {
        const unsigned low = rest & (0u - rest);
        if ((im >> i) & 1u) out |= low;
        rest &= rest - 1;
    }
    return out;
}

// Per-lane search: over items 0 .. len-1 in order, the first whose running
// sum of val(i) exceeds q (-1 if none), `before` the running sum before it.
// Items are loaded NW at a time so that their loads are in flight together.
template <int NW, typename V, typename F>
__device__ __forceinline__ int lane_first_exceeding(int len, V q, F val, V &before)
{
    V run = 0;
    for (int b = 0; b < len; b += NW) {
        V v[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) v[i] = b + i < len ? val(b + i) : (V)0;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            if (b + i < len && run + v[i] > q) { before = run; return b + i; }
            run += v[i];
        }
    }
    return -1;
}

// The first index i in [lo, hi) with pred(i) true, for a predicate that is
// false then true along the range (hi if it is never true).  K = 1: binary
// search; K > 1: K probes per round, evenly spaced, all loads in flight
// together (about log_{K+1} of the range in dependent rounds).  on_probe()
// runs once per evaluated probe.
template <int K, typename P, typename F>
__device__ __forceinline__ int64_t first_true(int64_t lo, int64_t hi, P pred, F on_probe)
{
    if constexpr (K == 1) {
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            on_probe();
            if (pred(mid)) hi = mid; else lo = mid + 1;
        }
        return lo;
    } else {
        while (hi - lo > K) {
            const int64_t step = (hi - lo) / (K + 1);
            bool t[K];
#pragma unroll
            for (int i = 0; i < K; ++i) { t[i] = pred(lo + (i + 1) * step); on_probe(); }
            int64_t nlo = lo + K * step + 1, nhi = hi;
#pragma unroll
            for (int i = K - 1; i >= 0; --i)
                if (t[i]) { nhi = lo + (i + 1) * step; nlo = i ? lo + i * step + 1 : lo; }
            lo = nlo;
            hi = nhi;
        }
        bool t[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            t[i] = lo + i < hi ? pred(lo + i) : true;
            if (lo + i < hi) on_probe();
        }
#pragma unroll
        for (int i = K - 1; i >= 0; --i)
            if (t[i]) hi = lo + i;
        return hi;
    }
}

// Byte counts of the sampler's accesses, compiled in only when CNT: rb the
// bytes of the data items, rs the same accesses in 32-byte sectors (32 bytes
// per random access, contiguous runs by their bytes).
#define MC_COUNT(item, sector)           \
    do {                                 \
        if constexpr (CNT) {             \
            rb += (uint64_t)(item);      \
            rs += (uint64_t)(sector);    \
        }                                \
    } while (0)

// Up to NQ adjacency tests at once (binary search of the shorter list),
// advancing all searches one level per round so their loads overlap.
template <int NQ = 4, bool CNT = false>
__device__ __forceinline__ void adjacent4(const int64_t *row_ptr, const uint32_t *col, const uint32_t *qa,
                                          const uint32_t *qb, int nq, bool *out, uint64_t &rb, uint64_t &rs)
{
    int64_t lo[NQ], hi[NQ], end[NQ];
    uint32_t key[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        if (i < nq) {
            uint32_t x = qa[i], y = qb[i];
            const int64_t dx = row_ptr[x + 1] - row_ptr[x], dy = row_ptr[y + 1] - row_ptr[y];
            if (dy < dx) { const uint32_t t = x; x = y; y = t; }
            lo[i] = row_ptr[x];
            hi[i] = row_ptr[x + 1];
            end[i] = hi[i];
            key[i] = y;
            MC_COUNT(32 + 4, 64 + 32);  // both degrees, the final probe
        } else {
            lo[i] = hi[i] = end[i] = 0;
            key[i] = 0;
        }
    }
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int i = 0; i < NQ; ++i)
            if (lo[i] < hi[i]) {
                const int64_t mid = (lo[i] + hi[i]) >> 1;
                if (col[mid] < key[i]) lo[i] = mid + 1; else hi[i] = mid;
                MC_COUNT(4, 32);
                more |= lo[i] < hi[i];
            }
    }
#pragma unroll
    for (int i = 0; i < NQ; ++i) out[i] = i < nq && lo[i] < end[i] && col[lo[i]] == key[i];
}

// The same tests for pairs of a sample's nodes whose adjacency offsets
// (rlo, degree rdg) were loaded once per node: qa, qb index nodes[].
template <int NQ, bool CNT>
__device__ __forceinline__ void adjacent_nodes(const uint32_t *col, const int64_t *rlo, const uint32_t *rdg,
                                               const uint32_t *nodes, const uint32_t *qa, const uint32_t *qb,
                                               int nq, bool *out, uint64_t &rb, uint64_t &rs)
{
    int64_t lo[NQ], hi[NQ], end[NQ];
    uint32_t key[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        if (i < nq) {
            uint32_t x = qa[i], y = qb[i];
            if (rdg[y] < rdg[x]) { const uint32_t t = x; x = y; y = t; }
            lo[i] = rlo[x];
            hi[i] = lo[i] + rdg[x];
            end[i] = hi[i];
            key[i] = nodes[y];
            MC_COUNT(4, 32);  // the final probe
        } else {
            lo[i] = hi[i] = end[i] = 0;
            key[i] = 0;
        }
    }
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int i = 0; i < NQ; ++i)
            if (lo[i] < hi[i]) {
                const int64_t mid = (lo[i] + hi[i]) >> 1;
                if (col[mid] < key[i]) lo[i] = mid + 1; else hi[i] = mid;
                MC_COUNT(4, 32);
                more |= lo[i] < hi[i];
            }
    }
#pragma unroll
    for (int i = 0; i < NQ; ++i) out[i] = i < nq && lo[i] < end[i] && col[lo[i]] == key[i];
}

// Lane-per-sample sampler: the 32 lanes of a warp draw 32 samples and walk
// their h-1 decomposition steps in lockstep (every h-treelet has h-1 internal
// decomposition nodes).  A lane does its own scalar work, short scans and
// binary searches (a hub's chunk by the prefix sums of its chunks).  CT: the
// tables' count type; V: the type of the descent's weights, draws and
// running sums (64 bits when every level total leaves room for beta, else
// 128 bits).

// Occupancy target: 6 blocks of 256 per SM for 64-bit counts, 4 for 128-bit
// ones (their wider state spills less; measured faster on both workloads).
// LAT (launches too small to fill the GPU, e.g. the batches of AGS): no
// register cap, 16 items of a scan and 8 adjacency searches in flight per
// lane, so each sample's chain of dependent loads is shorter.  The samples
// are the same in both modes.
template <typename CT, typename V, bool PK, bool LAT, bool CNT>
__global__ void __launch_bounds__(256, LAT ? 1 : (sizeof(CT) == 16 ? 4 : 6))
    sample_kernel(const __grid_constant__ SampleArgs a)
{
    constexpr int NW = LAT ? 16 : 4;  // items of a scan in flight
    constexpr int NQ = LAT ? 8 : 4;   // adjacency searches in flight
    constexpr int KS = LAT ? 8 : 1;   // probes per round of the root and hub chunk searches
    extern __shared__ unsigned int s_hist[];
    __shared__ SampleSmem sm;
    for (int i = threadIdx.x; i < (1 << (MAXK - 1)); i += blockDim.x) sm.crank[i] = a.crank[i];
    for (int i = threadIdx.x; i < MAXK * 36; i += blockDim.x) (&sm.unrank[0][0])[i] = (&a.unrank[0][0])[i];
    if (a.hist)
        for (int i = threadIdx.x; i < a.ncls; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int h = a.h;
    const int CB = (int)sizeof(CT);
    bool bad = false;
    uint64_t rb = 0, rs = 0;  // byte counts (CNT): data items, 32-byte sectors
    // a warp's next batch of 32 samples: from the shared counter (the warps
    // that draw cheap samples take more batches, so they end together), or
    // every nwarps-th batch
    auto take = [&](int64_t after) -> int64_t {
        if (!a.next) return after < 0 ? warp * 32 : after + nwarps * 32;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(a.next, 32ull);
        return (int64_t)__shfl_sync(0xffffffffu, b, 0);
    };
    for (int64_t base = take(-1); base < a.count; base = take(base)) {
        const int64_t sid = base + lane;
        bool ok = sid < a.count;
        uint64_t index = a.first_index + (uint64_t)sid;
        const u128 *prefix = a.prefix;
        const uint32_t *bucket = a.bucket;
        u128 R = a.R, Xbase = a.Xbase, D = a.D;
        uint64_t allow0 = a.allow0, allow1 = a.allow1;
        if (a.nseg > 0 && ok) {  // the part this sample falls in
            int g = 0;
            while (g + 1 < a.nseg && sid >= a.seg[g].end) ++g;
            const SampleSeg &sg = a.seg[g];
            index = sg.first_index + (uint64_t)(sid - (g ? a.seg[g - 1].end : 0));
            prefix = sg.prefix;
            bucket = sg.bucket;
            R = sg.R;
            Xbase = sg.Xbase;
            D = sg.D;
            allow0 = sg.allow0;
            allow1 = sg.allow1;
        }
        // ---- root: X = uniform(R); v = first node with prefix[v] > X, found
        // by binary search inside the bucket of X
        V X = 0;
        uint32_t v = 0;
        if (ok && !draw_below(a.seed, index, 0, (V)R, X)) { ok = false; bad = true; }
        X += (V)Xbase;  // a node range: the draw lands inside its part of the prefix
        if (ok) {
            const uint64_t bk = (uint64_t)(X / (V)D);
            const int64_t blo = bucket[bk], bhi = bucket[bk + 1];
            MC_COUNT(8, 32);
            const int64_t lo = first_true<KS>(
                blo, bhi, [&](int64_t i) { return prefix[i] > (u128)X; }, [&] { MC_COUNT(16, 32); });
            MC_COUNT(32, 32);  // the check below and prefix[v - 1]
            v = (uint32_t)lo;
            if (!(prefix[v] > (u128)X)) { ok = false; bad = true; }
        }
        // ---- entry of v's level-h row, in (shape id, colour mask) order
        int s0 = 0, cv0 = 0;
        unsigned C0 = 0;
        if (ok) {
            const V rem = X - (v ? (V)prefix[v - 1] : (V)0);
            const int Bc = a.Bc[h], Rh = a.R_[h];
            V bf;
            // e runs in (shape id, colour mask) order; the row is set-major
            const int found = lane_first_exceeding<NW, V>(a.Wc[h], rem, [&](int e) -> V {
                const int sh = e / Bc;
                const bool al = sh < 64 ? (allow0 >> sh) & 1 : (allow1 >> (sh - 64)) & 1;
                MC_COUNT(al ? CB : 0, al ? CB : 0);  // one contiguous row
                return al ? (V)c_at<CT, PK>(a, h, v, (e - sh * Bc) * Rh + sh) : (V)0;
            }, bf);
            if (found < 0) { ok = false; bad = true; }
            else {
                cv0 = a.colors[v];
                s0 = found / Bc;
                C0 = (1u << cv0) | insert_colour_gap(sm.unrank[h - 1][found % Bc], cv0);
            }
        }
        // ---- descent: decomposition nodes in pre-order (T' before T'')
        int stg[MAXK], stc[MAXK], sp = 0, nn = 0, ne = 0;
        unsigned stC[MAXK];
        uint32_t stx[MAXK], nodes[MAXK], ea[MAXK], eb[MAXK];
        if (ok) { stg[0] = a.first[h] + s0; stC[0] = C0; stx[0] = v; stc[0] = cv0; sp = 1; }
        for (uint32_t step = 1; step < (uint32_t)h; ++step) {
            int g = 0, cx = 0;
            unsigned C = 0;
            uint32_t x = 0;
            if (ok) {  // leaves on top of the stack are sample nodes
                for (;;) {
                    if (sp <= 0 || nn >= MAXK) { ok = false; bad = true; break; }
                    --sp;
                    g = stg[sp]; C = stC[sp]; x = stx[sp]; cx = stc[sp];
                    if (a.sz[g] > 1) break;
                    nodes[nn++] = x;
                }
            }
            int ga = 0, gb = 0, hb = 1, sbase = 0, sidx = 0, chunk0 = -1;
            unsigned C1 = 0, C2 = 0;
            int64_t e0 = 0, e1 = 0, nch = 0;
            CT q = 0;
            if (ok) {
                ga = a.lft[g]; gb = a.rgt[g]; hb = a.sz[gb];
                MC_COUNT(16 + 4 + CB, 96);  // row offsets, first chunk, c(T_C, x)
                e0 = a.row_ptr[x];
                e1 = a.row_ptr[x + 1];
                chunk0 = a.node_chunk0[x];
                const V W = (V)a.beta[g] * count_at<CT, V, PK>(a, sm, g, C, x, cx);
                V Y = 0;
                if (!draw_below(a.seed, index, step, W, Y)) { ok = false; bad = true; }
                if (ok) {
                    // block of C'' (ascending mask), weights c(T'_{C\C''}, x) S(T'', C'', x)
                    const unsigned rest = C & ~(1u << cx);
                    const int nr = __popc(rest);
                    int nsub = 1;
                    for (int i = 1; i <= hb; ++i) nsub = nsub * (nr - hb + i) / i;
                    sbase = a.loc[gb];
                    const int Rb = a.R_[hb];
                    V before;
                    const int blk = lane_first_exceeding<NW, V>(nsub, Y, [&](int i) -> V {
                        const unsigned c2 = deposit(sm.unrank[hb][i], rest);
                        MC_COUNT(2 * CB, 64);
                        return count_at<CT, V, PK>(a, sm, ga, C & ~c2, x, cx) *
                               (V)s_at<CT, PK>(a, hb, x, sm.crank[drop_colour(c2, cx)] * Rb + sbase);
                    }, before);
                    if (blk < 0) { ok = false; bad = true; }
                    else {
                        C2 = deposit(sm.unrank[hb][blk], rest);
                        C1 = C & ~C2;
                        const V x1 = count_at<CT, V, PK>(a, sm, ga, C1, x, cx);
                        q = (CT)quotient(Y - before, x1);  // < S(T'', C'', x): fits CT
                        sidx = sm.crank[drop_colour(C2, cx)] * a.R_[hb] + sbase;
                        if (chunk0 >= 0) nch = (e1 - e0 + HUB_CHUNK - 1) / HUB_CHUNK;
                    }
                }
            }
            // ---- hub: the 64-neighbour chunk holding the answer, from the
            // inclusive prefix of its chunk sums (contiguous per hub and entry)
            // T'' one node: c(T''_{C''}, u) is 1 for the neighbours of the one
            // colour of C'' and 0 otherwise, so the answer is the (q+1)-th
            // neighbour of that colour in ascending id order: position q of
            // that colour's block in the colour-sorted adjacency
            const bool single = ok && hb == 1;
            const bool chunked = ok && !single && chunk0 >= 0;
            const CT *spp = nullptr;
            if (chunked) spp = (const CT *)a.Sp[hb] + (int64_t)chunk0 * a.Ws[hb] + (int64_t)sidx * nch;
            int64_t ci = -1;
            CT bc = 0;
            if (chunked) {
                // the first chunk whose inclusive prefix exceeds q: a binary
                // search of the hub's chunk prefix sums for this S entry
                const int64_t lo = first_true<KS>(
                    0, nch - 1, [&](int64_t i) { return spp[i] > q; }, [&] { MC_COUNT(CB, 32); });
                MC_COUNT(2 * CB, 32);
                if (spp[lo] > q) { ci = lo; bc = lo ? spp[lo - 1] : (CT)0; }
            }
            int64_t lo_e = e0, hi_e = e1;
            CT qq = q;
            if (chunked) {
                if (ci < 0) { ok = false; bad = true; }
                else {
                    lo_e = e0 + ci * HUB_CHUNK;
                    hi_e = min(e1, lo_e + HUB_CHUNK);
                    qq = q - bc;
                }
            }
            // ---- neighbour: first u (ascending) whose running sum of
            // c(T''_{C''}, u) exceeds qq (at most HUB_CHUNK neighbours)
            if (single) {
                const int col2 = __ffs(C2) - 1;
                const int32_t b0 = a.coff[(int64_t)x * (a.k + 1) + col2];
                const int32_t b1 = a.coff[(int64_t)x * (a.k + 1) + col2 + 1];
                MC_COUNT(8 + 4, 64);
                if ((uint64_t)q >= (uint64_t)(b1 - b0) || sp + 2 > MAXK || ne >= MAXK) { ok = false; bad = true; }
                else {
                    const uint32_t u = a.scol[e0 + b0 + (int64_t)q];
                    ea[ne] = x; eb[ne] = u; ++ne;
                    stg[sp] = gb; stC[sp] = C2; stx[sp] = u; stc[sp] = col2; ++sp;
                    stg[sp] = ga; stC[sp] = C1; stx[sp] = x; stc[sp] = cx; ++sp;
                }
            } else if (ok) {
                int64_t sel = -1;
                {
                    const int lb = a.loc[gb];
                    const int rcb = a.R_[hb];
                    CT bn;
                    const int r = lane_first_exceeding<NW, CT>((int)(hi_e - lo_e), qq, [&](int i) -> CT {
                        const int cu = a.ecol[lo_e + i];
                        MC_COUNT(1, 1);  // contiguous edge colours
                        if (!((C2 >> cu) & 1u)) return (CT)0;
                        MC_COUNT(4 + CB, 4 + 32);  // contiguous ids; the neighbour's row entry
                        const uint32_t u = a.col[lo_e + i];
                        return c_at<CT, PK>(a, hb, u, sm.crank[drop_colour(C2 & ~(1u << cu), cu)] * rcb + lb);
                    }, bn);
                    if (r >= 0) sel = lo_e + r;
                }
                if (sel < 0 || sp + 2 > MAXK || ne >= MAXK) { ok = false; bad = true; }
                else {
                    const uint32_t u = a.col[sel];
                    const int cu = a.ecol[sel];
                    ea[ne] = x; eb[ne] = u; ++ne;   // a treelet edge: adjacent for sure
                    stg[sp] = gb; stC[sp] = C2; stx[sp] = u; stc[sp] = cu; ++sp;
                    stg[sp] = ga; stC[sp] = C1; stx[sp] = x; stc[sp] = cx; ++sp;
                }
            }
        }
        if (ok) {  // remaining leaves
            while (sp > 0 && nn < MAXK) { --sp; nodes[nn++] = stx[sp]; }
            if (nn != h || sp != 0) { ok = false; bad = true; }
        }
        int cls = -1;
        if (ok) {
            for (int i = 1; i < h; ++i)
                for (int j = i; j > 0 && nodes[j - 1] > nodes[j]; --j) {
                    const uint32_t tmp = nodes[j]; nodes[j] = nodes[j - 1]; nodes[j - 1] = tmp;
                }
            // induced subgraph: the treelet's edges are known; the other pairs
            // are tested against the adjacency lists, four at a time
            const int P = h * (h - 1) / 2;
            uint32_t word = 0, known = 0;
            for (int t = 0; t < ne; ++t) {
                int i = 0, j = 0;
                for (int p = 0; p < h; ++p) {
                    if (nodes[p] == ea[t]) i = p;
                    if (nodes[p] == eb[t]) j = p;
                }
                if (i > j) { const int tmp = i; i = j; j = tmp; }
                known |= 1u << pair_pos(h, i, j);
            }
            word = known;
            int64_t rlo[MAXK];  // adjacency offsets and degrees, loaded once per node
            uint32_t rdg[MAXK];
            for (int i = 0; i < h; ++i) {
                rlo[i] = a.row_ptr[nodes[i]];
                rdg[i] = (uint32_t)(a.row_ptr[nodes[i] + 1] - rlo[i]);
                MC_COUNT(16, 32);
            }
            uint32_t qa[NQ], qb[NQ];
            int qp[NQ], nq = 0;
            for (int p = 0; p < P; ++p) {
                const int i = a.pi[p], j = a.pj[p];
                const int bit = pair_pos(h, i, j);
                if ((known >> bit) & 1u) continue;
                qa[nq] = i; qb[nq] = j; qp[nq] = bit; ++nq;
                if (nq == NQ || p == P - 1) {
                    bool r4[NQ];
                    adjacent_nodes<NQ, CNT>(a.col, rlo, rdg, nodes, qa, qb, nq, r4, rb, rs);
                    for (int t = 0; t < nq; ++t)
                        if (r4[t]) word |= 1u << qp[t];
                    nq = 0;
                }
            }
            if (nq) {
                bool r4[NQ];
                adjacent_nodes<NQ, CNT>(a.col, rlo, rdg, nodes, qa, qb, nq, r4, rb, rs);
                for (int t = 0; t < nq; ++t)
                    if (r4[t]) word |= 1u << qp[t];
            }
            cls = a.lut[word];
            MC_COUNT(2, 32);
            if (cls == 0xffff) { cls = -1; bad = true; }
            if (a.nodes) for (int i = 0; i < h; ++i) a.nodes[sid * h + i] = nodes[i];
            if (a.roots) a.roots[sid] = v;
            if (a.shapes) a.shapes[sid] = s0;
            {
                const int ob = (a.nodes ? 4 * h : 0) + (a.roots ? 4 : 0) + (a.shapes ? 4 : 0) + (a.classes ? 4 : 0);
                MC_COUNT(ob, ob);
            }
            if (a.hist && cls >= 0) atomicAdd(&s_hist[cls], 1u);
        }
        if (sid < a.count && a.classes) a.classes[sid] = cls;
    }
    if (bad) atomicOr(a.err, SERR_SEARCH);
    if (CNT && a.bytes) {
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            rb += __shfl_xor_sync(0xffffffffu, rb, d);
            rs += __shfl_xor_sync(0xffffffffu, rs, d);
        }
        if (lane == 0) {
            atomicAdd(a.bytes, (unsigned long long)rb);
            atomicAdd(a.bytes + 1, (unsigned long long)rs);
        }
    }
    if (a.hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < a.ncls; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&a.hist[i], (unsigned long long)s_hist[i]);
    }
}

// Uniform estimator (Section 2.2): g_i = ((t * hits_i) / (sigma_i * N)) * (1/p),
// one correctly rounded operation at a time.
__global__ void uniform_estimate_kernel(const unsigned long long *hits, const int64_t *sigma, int ncls,
                                        u128 t, int64_t N, double inv_p, double *est)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncls) return;
    if (sigma[i] <= 0) { est[i] = 0.0; return; }  // graphlets no counted tree spans
    const double td = u128_to_double(t);
    const double num = __dmul_rn(td, __ull2double_rn(hits[i]));
    const double den = __dmul_rn(__ll2double_rn(sigma[i]), __ll2double_rn(N));
    est[i] = __dmul_rn(__ddiv_rn(num, den), inv_p);
}

// ---------------------------------------------------------------------------
// Uncoloured star sampling (Section 3.3.2).  Node weights C(d_v, h-1), their
// inclusive prefix, then one thread per sample: the centre by a binary
// search of the prefix, the leaves by sequential selection without
// replacement (the x-th untaken position, x = uniform(d_v - s)).
// ---------------------------------------------------------------------------
constexpr uint32_t STAR_STEP = 16;

// q = x / d for a small divisor, by 32-bit long division
__device__ __forceinline__ u128 div_small(u128 x, uint32_t d)
{
    u128 q = 0;
    uint64_t r = 0;
    for (int i = 3; i >= 0; --i) {
        const uint64_t cur = (r << 32) | (uint32_t)(x >> (32 * i));
        q |= (u128)(cur / d) << (32 * i);
        r = cur % d;
    }
    return q;
}

__global__ void star_weights_kernel(const int64_t *__restrict__ row_ptr, int64_t n, int r, u128 *__restrict__ w,
                                    int *err)
{
    bool ovf = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        u128 c = d >= r ? 1 : 0;
        // C(d, r) = prod_{i=1..r} (d - r + i) / i; each partial product is
        // i * C(d - r + i, i), so every division is exact
        for (int i = 1; i <= r && c; ++i) {
            u128 p;
            ovf |= mul_ovf(c, (u128)(d - r + i), p);
            c = div_small(p, (uint32_t)i);
        }
        w[v] = c;
    }
    if (ovf) atomicOr(err, 1);
}

struct StarArgs {
    const int64_t *row_ptr;
    const uint32_t *col;
    const u128 *prefix;
    const uint32_t *bucket;  // first node whose prefix exceeds b * D, b = 0..nb
    u128 D;
    int64_t n;
    u128 S;
    int h;
    uint64_t seed, first_index;
    int64_t count;
    const uint16_t *lut;
    uint32_t *nodes, *centres;
    int32_t *classes;
    unsigned long long *hist;
    int *err;
};

// V: the type of the centre draw (64 bits when S < 2^64, the same value as
// the 128-bit draw)
template <typename V>
__global__ void __launch_bounds__(256) star_kernel(const __grid_constant__ StarArgs a)
{
    bool bad = false;
    const int h = a.h;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = a.first_index + (uint64_t)i;
        V X;
        if (!draw_below(a.seed, idx, STAR_STEP, (V)a.S, X)) { bad = true; continue; }
        // the first node whose prefix exceeds X lies in X's bucket
        const uint64_t bk = (uint64_t)(X / (V)a.D);
        int64_t lo = a.bucket[bk], hi = a.bucket[bk + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (a.prefix[mid] > (u128)X) hi = mid; else lo = mid + 1;
        }
        const int64_t v = lo, e0 = a.row_ptr[v];
        if (!(a.prefix[v] > (u128)X)) { bad = true; continue; }
        const uint64_t d = (uint64_t)(a.row_ptr[v + 1] - e0);
        if (d < (uint64_t)(h - 1)) { bad = true; continue; }
        uint64_t pos[MAXK];
        int taken = 0;
        for (int s = 0; s < h - 1; ++s) {
            uint64_t x;
            if (!draw_below(a.seed, idx, STAR_STEP + 1 + (uint32_t)s, d - (uint64_t)s, x)) { bad = true; break; }
            int j = 0;
            while (j < taken && pos[j] <= x) { ++x; ++j; }  // skip the positions taken
            for (int q = taken; q > j; --q) pos[q] = pos[q - 1];
            pos[j] = x;
            ++taken;
        }
        if (taken != h - 1) continue;
        // the centre among its leaves, ascending (leaves ascend with position)
        uint32_t nd[MAXK];
        int m = 0;
        bool placed = false;
        const uint32_t c = (uint32_t)v;
        for (int s = 0; s < h - 1; ++s) {
            const uint32_t u = a.col[e0 + (int64_t)pos[s]];
            if (!placed && c < u) { nd[m++] = c; placed = true; }
            nd[m++] = u;
        }
        if (!placed) nd[m++] = c;
        // centre-leaf pairs are edges; leaf-leaf pairs by binary search,
        // four searches in flight
        uint32_t word = 0, qa[4], qb[4];
        int qp[4], nq = 0;
        uint64_t rb = 0, rs = 0;
        for (int x = 0; x < h; ++x)
            for (int y = x + 1; y < h; ++y) {
                if (nd[x] == c || nd[y] == c) { word |= 1u << pair_pos(h, x, y); continue; }
                qa[nq] = nd[x]; qb[nq] = nd[y]; qp[nq] = pair_pos(h, x, y); ++nq;
                if (nq == 4) {
                    bool r4[4];
                    adjacent4(a.row_ptr, a.col, qa, qb, nq, r4, rb, rs);
                    for (int q = 0; q < nq; ++q) if (r4[q]) word |= 1u << qp[q];
                    nq = 0;
                }
            }
        if (nq) {
            bool r4[4];
            adjacent4(a.row_ptr, a.col, qa, qb, nq, r4, rb, rs);
            for (int q = 0; q < nq; ++q) if (r4[q]) word |= 1u << qp[q];
        }
        const int cls = a.lut[word];
        if (cls == 0xffff) bad = true;
        if (a.nodes) for (int x = 0; x < h; ++x) a.nodes[i * h + x] = nd[x];
        if (a.centres) a.centres[i] = c;
        if (a.classes) a.classes[i] = cls == 0xffff ? -1 : cls;
        if (a.hist && cls != 0xffff) atomicAdd(&a.hist[cls], 1ull);
    }
    if (bad) atomicOr(a.err, 2);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void fill_sample_args(SampleArgs &a, const mc_tables *t, int h)
{
    const ShapeCatalog &cat = shape_catalog();
    const mc_graph *g = t->g;
    a = SampleArgs{};
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.colors = t->colors;
    a.ecol = t->ecol;
    a.scol = t->scol;
    a.coff = t->coff;
    a.n = g->n;
    a.node_chunk0 = g->node_chunk0;
    for (int i = 1; i <= t->k; ++i) {
        a.c[i] = t->c[i];
        a.S[i] = t->S[i];
        a.pc[i] = t->pc[i];
        a.ps[i] = t->ps[i];
        a.Sp[i] = t->Sp[i];
        a.Bc[i] = t->geo.Bc[i];
        a.Bs[i] = t->geo.Bs[i];
        a.Wc[i] = t->geo.Wc[i];
        a.Ws[i] = t->geo.Ws[i];
        a.R_[i] = cat.r[i];
    }
    a.k = t->k;
    a.h = h;
    for (int i = 0; i <= MAXK + 1; ++i) a.first[i] = cat.first[std::min(i, MAXK + 1)];
    for (int gid = 0; gid < cat.first[t->k + 1]; ++gid) {
        const Shape &s = cat.shapes[gid];
        a.sz[gid] = (uint8_t)s.size;
        a.loc[gid] = (uint8_t)s.local;
        a.lft[gid] = (uint8_t)std::max(s.left, 0);
        a.rgt[gid] = (uint8_t)std::max(s.right, 0);
        a.beta[gid] = (uint8_t)s.beta;
    }
    if (t->skip_round) {  // level k descends by its balanced decompositions
        const Programs &P = programs(t->k, true);
        for (int gid = cat.first[t->k]; gid < cat.first[t->k + 1]; ++gid) {
            a.lft[gid] = (uint8_t)std::max(P.bal_left[gid], 0);
            a.rgt[gid] = (uint8_t)std::max(P.bal_right[gid], 0);
            a.beta[gid] = (uint8_t)P.bal_beta[gid];
        }
    }
    for (unsigned m = 0; m < (1u << (t->k - 1)); ++m) a.crank[m] = (uint8_t)colex_rank(m);
    for (int m = 0; m < MAXK; ++m)
        for (int i = 0; i < binom(MAXK - 1, m); ++i) a.unrank[m][i] = (uint8_t)colex_unrank(m, i);
    int p = 0;
    for (int i = 0; i < h; ++i)
        for (int j = i + 1; j < h; ++j) { a.pi[p] = (uint8_t)i; a.pj[p] = (uint8_t)j; ++p; }
}

struct RootIndex {
    const u128 *prefix = nullptr;
    u128 R = 0;      // total of the node range
    u128 base = 0;   // prefix before the range
    u128 Rall = 0;   // total of all nodes
    const uint32_t *bucket = nullptr;
    u128 D = 1;
};

void launch_row_totals(const mc_tables *t, int h, uint64_t allow0, uint64_t allow1, u128 *tot, int *err,
                       cudaStream_t s);
void launch_treelet_totals(const mc_tables *t, int h, u128 *tot, int *err, cudaStream_t s);
void build_buckets(const u128 *prefix, int64_t n, int64_t nb, u128 *dD, uint32_t *start, cudaStream_t s);
int64_t bucket_count(int64_t n);

// Restrict a root index to the nodes [lo, hi) (hi <= 0: all nodes).
static void restrict_range(RootIndex &ri, int64_t n, int64_t lo, int64_t hi, cudaStream_t s)
{
    ri.Rall = ri.R;
    if (hi <= 0 && lo <= 0) return;
    if (hi <= 0) hi = n;
    MC_REQUIRE(lo >= 0 && lo < hi && hi <= n, "node range out of bounds");
    u128 top = 0, base = 0;
    MC_CUDA(cudaMemcpyAsync(&top, ri.prefix + (hi - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
    if (lo > 0) MC_CUDA(cudaMemcpyAsync(&base, ri.prefix + (lo - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    ri.base = base;
    ri.R = top - base;
}

static RootIndex root_index(const mc_tables *t, int h, int unrooted, Arena &scratch, int *err, cudaStream_t s,
                            uint64_t &allow0, uint64_t &allow1, int64_t lo = 0, int64_t hi = 0)
{
    const ShapeCatalog &cat = shape_catalog();
    allow0 = allow1 = 0;
    for (int i = 0; i < cat.r[h]; ++i)
        if (unrooted < 0 || cat.shapes[cat.gid(h, i)].unrooted == unrooted) {
            if (i < 64) allow0 |= 1ull << i; else allow1 |= 1ull << (i - 64);
        }
    RootIndex ri;
    if (unrooted < 0) {
        ensure_level_index(t, h, s);
        ri.prefix = t->prefix[h];
        ri.R = t->R[h];
        ri.bucket = t->bucket[h];
        ri.D = t->bucketD[h];
        restrict_range(ri, t->g->n, lo, hi, s);
        return ri;
    }
    const int64_t n = t->g->n;
    u128 *p = scratch.get<u128>((size_t)n);
    uint32_t *bk = scratch.get<uint32_t>((size_t)t->nbucket + 1);
    u128 *dD = scratch.get<u128>(1);
    launch_row_totals(t, h, allow0, allow1, p, err, s);
    inclusive_scan_u128(p, n, err, scratch, s);
    build_buckets(p, n, t->nbucket, dD, bk, s);
    if (n) {
        MC_CUDA(cudaMemcpyAsync(&ri.R, p + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(&ri.D, dD, sizeof(u128), cudaMemcpyDeviceToHost, s));
    }
    MC_CUDA(cudaStreamSynchronize(s));
    ri.prefix = p;
    ri.bucket = bk;
    restrict_range(ri, n, lo, hi, s);
    return ri;
}

// The root index of every unrooted treelet of level h (what root_index gives
// for each j), with dense tables from one pass over the level's rows and one
// synchronisation.
static std::vector<RootIndex> treelet_root_indexes(const mc_tables *t, int h, Arena &scratch, int *err,
                                                   cudaStream_t s,
                                                   std::vector<std::pair<uint64_t, uint64_t>> &allows,
                                                   int64_t lo, int64_t hi)
{
    const ShapeCatalog &cat = shape_catalog();
    const int nu = cat.n_unrooted[h];
    std::vector<RootIndex> ris((size_t)nu);
    allows.assign((size_t)nu, {0, 0});
    if (t->packed) {
        for (int j = 0; j < nu; ++j)
            ris[j] = root_index(t, h, j, scratch, err, s, allows[j].first, allows[j].second, lo, hi);
        return ris;
    }
    for (int i = 0; i < cat.r[h]; ++i) {
        auto &al = allows[(size_t)cat.shapes[cat.gid(h, i)].unrooted];
        if (i < 64) al.first |= 1ull << i; else al.second |= 1ull << (i - 64);
    }
    const int64_t n = t->g->n;
    u128 *p = scratch.get<u128>((size_t)n * nu);
    u128 *dD = scratch.get<u128>((size_t)nu);
    launch_treelet_totals(t, h, p, err, s);
    for (int j = 0; j < nu; ++j) {
        u128 *pj = p + (size_t)j * n;
        uint32_t *bk = scratch.get<uint32_t>((size_t)t->nbucket + 1);
        inclusive_scan_u128(pj, n, err, scratch, s);
        build_buckets(pj, n, t->nbucket, dD + j, bk, s);
        if (n) {
            MC_CUDA(cudaMemcpyAsync(&ris[j].R, pj + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(&ris[j].D, dD + j, sizeof(u128), cudaMemcpyDeviceToHost, s));
        }
        ris[j].prefix = pj;
        ris[j].bucket = bk;
    }
    MC_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < nu; ++j) restrict_range(ris[j], n, lo, hi, s);
    return ris;
}

static void launch_sampler(const mc_tables *t, SampleArgs &a, cudaStream_t s)
{
    // a launch that leaves most SMs idle runs the latency mode (dense tables)
    // in blocks of 64, spread over more SMs
    const bool lat = !t->packed && a.count <= (int64_t)sm_count() * 256;
    const int block = lat ? 64 : 256;
    const size_t smem = a.hist ? (size_t)a.ncls * sizeof(unsigned int) : 0;
    // one wave of resident blocks: the grid-stride loop then keeps every
    // warp busy until the samples run out
    // 64-bit descent arithmetic is exact when 8 R < 2^64: every weight is at
    // most beta (<= 7) times a count of the level, every running sum at most
    // a level total
    const bool narrow = t->bits == 64 && ((a.R + a.Xbase) >> 61) == 0;
    // byte counting (profiling) runs its own instantiation of the dense,
    // throughput-mode kernel, so uncounted launches carry none of its work
    const bool cnt = a.bytes != nullptr && !t->packed && !lat;
    if (!cnt) a.bytes = nullptr;
    auto kern = t->packed ? (t->bits == 64 ? (narrow ? sample_kernel<uint64_t, uint64_t, true, false, false>
                                                     : sample_kernel<uint64_t, u128, true, false, false>)
                                           : sample_kernel<u128, u128, true, false, false>)
              : lat ? (t->bits == 64 ? (narrow ? sample_kernel<uint64_t, uint64_t, false, true, false>
                                               : sample_kernel<uint64_t, u128, false, true, false>)
                                     : sample_kernel<u128, u128, false, true, false>)
              : cnt ? (t->bits == 64 ? (narrow ? sample_kernel<uint64_t, uint64_t, false, false, true>
                                               : sample_kernel<uint64_t, u128, false, false, true>)
                                     : sample_kernel<u128, u128, false, false, true>)
                    : (t->bits == 64 ? (narrow ? sample_kernel<uint64_t, uint64_t, false, false, false>
                                               : sample_kernel<uint64_t, u128, false, false, false>)
                                     : sample_kernel<u128, u128, false, false, false>);
    int per_sm = 0;
    MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (a.count + block - 1) / block;  // one sample per thread
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (smem > 48 * 1024)
        MC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MC_LAUNCH("sample", s, kern<<<(unsigned)grid, block, smem, s>>>(a));
}

// The sampler's batch counter, zeroed on the stream.
static unsigned long long *batch_counter(Arena &scratch, cudaStream_t s)
{
    unsigned long long *c = scratch.get<unsigned long long>(1);
    MC_CUDA(cudaMemsetAsync(c, 0, sizeof(unsigned long long), s));
    return c;
}

// While profiling is on, the sampler counts the bytes of the data items it
// reads and writes into a device counter from `scratch`; the count is added
// to the profile after the launch (one more synchronisation).
static unsigned long long *sample_byte_counter(Arena &scratch, cudaStream_t s)
{
    if (!prof_counting()) return nullptr;
    unsigned long long *c = scratch.get<unsigned long long>(2);
    MC_CUDA(cudaMemsetAsync(c, 0, 2 * sizeof(unsigned long long), s));
    return c;
}

// The sampler's counts: "sample" the bytes of the data items, "sample
// sectors" the same accesses at 32 bytes per random access.
static void report_sample_bytes(const unsigned long long *c, cudaStream_t s)
{
    if (!c) return;
    unsigned long long v[2] = {0, 0};
    MC_CUDA(cudaMemcpyAsync(v, c, sizeof(v), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    prof_add_bytes("sample", (int64_t)v[0]);
    prof_add_bytes("sample sectors", (int64_t)v[1]);
}

static double inv_colourful_prob(int k, int h)
{
    double num = 1.0, den = 1.0;
    for (int i = 0; i < h; ++i) num *= (double)k;
    for (int i = 1; i <= k - h; ++i) num *= (double)i;
    for (int i = 1; i <= k; ++i) den *= (double)i;
    return num / den;
}

// 1 / p for the biased colouring (lambda = L / 2^32): an h-node set is
// colourful with probability h! e_h(p_0, lambda, ..., lambda) =
// h! (C(k-1,h) lambda^h + C(k-1,h-1) lambda^(h-1) p_0), p_0 = 1 - (k-1) lambda;
// lambda and p_0 are exact doubles, the rest is evaluated in this order.
static double inv_colourful_prob_biased(int k, int h, uint32_t L)
{
    if (L == 0) return inv_colourful_prob(k, h);
    const double lam = (double)L / 4294967296.0;
    const double p0 = (double)(4294967296ull - (uint64_t)(k - 1) * L) / 4294967296.0;
    double lh1 = 1.0;
    for (int i = 0; i < h - 1; ++i) lh1 *= lam;
    double fact = 1.0;
    for (int i = 2; i <= h; ++i) fact *= (double)i;
    const double p = fact * ((double)binom(k - 1, h) * (lh1 * lam) + (double)binom(k - 1, h - 1) * (lh1 * p0));
    return 1.0 / p;
}

}  // namespace mc

using namespace mc;

extern "C" int mc_num_shapes(int h)
{
    if (h < 1 || h > MAXK) return -1;
    return shape_catalog().r[h];
}

extern "C" int mc_num_unrooted(int h)
{
    if (h < 1 || h > MAXK) return -1;
    return shape_catalog().n_unrooted[h];
}

extern "C" int mc_num_classes(int h)
{
    int out = -1;
    mc_status st = guarded([&] { out = (int)class_catalog(h)->codes.size(); });
    return st == MC_OK ? out : -1;
}

extern "C" mc_status mc_shape_info(int h, uint32_t *code, int32_t *unrooted, int32_t *beta, int32_t *left,
                                   int32_t *right)
{
    return guarded([&] {
        MC_REQUIRE(h >= 1 && h <= MAXK, "h must be in 1..8");
        const ShapeCatalog &cat = shape_catalog();
        for (int i = 0; i < cat.r[h]; ++i) {
            const Shape &s = cat.shapes[cat.gid(h, i)];
            if (code) code[i] = s.code;
            if (unrooted) unrooted[i] = s.unrooted;
            if (beta) beta[i] = s.beta;
            if (left) left[i] = s.left < 0 ? -1 : cat.shapes[s.left].local;
            if (right) right[i] = s.right < 0 ? -1 : cat.shapes[s.right].local;
        }
    });
}

extern "C" mc_status mc_skip_round_info(int k, int32_t *beta, int32_t *left_size, int32_t *left,
                                        int32_t *right_size, int32_t *right, int32_t *copies)
{
    return guarded([&] {
        MC_REQUIRE(k >= 4 && k <= MAXK, "k must be in 4..8");
        const ShapeCatalog &cat = shape_catalog();
        const Programs &P = programs(k, true);
        for (int i = 0; i < cat.r[k]; ++i) {
            const int g = cat.gid(k, i);
            const int l = P.bal_left[g], r = P.bal_right[g];
            if (beta) beta[i] = l < 0 ? -1 : P.bal_beta[g];
            if (left_size) left_size[i] = l < 0 ? -1 : cat.shapes[l].size;
            if (left) left[i] = l < 0 ? -1 : cat.shapes[l].local;
            if (right_size) right_size[i] = r < 0 ? -1 : cat.shapes[r].size;
            if (right) right[i] = r < 0 ? -1 : cat.shapes[r].local;
        }
        if (copies)
            for (int j = 0; j < cat.n_unrooted[k]; ++j) copies[j] = P.copies[j];
    });
}

extern "C" mc_status mc_class_codes(int h, uint32_t *codes)
{
    return guarded([&] {
        MC_REQUIRE(codes, "codes is NULL");
        const ClassCatalog *cc = class_catalog(h);
        std::copy(cc->codes.begin(), cc->codes.end(), codes);
    });
}

extern "C" mc_status mc_sigma(int h, int64_t *sigma_i, int64_t *sigma_ij)
{
    return guarded([&] {
        const ClassCatalog *cc = class_catalog_sigma(h);
        if (sigma_i) std::copy(cc->sigma_i.begin(), cc->sigma_i.end(), sigma_i);
        if (sigma_ij) std::copy(cc->sigma_ij.begin(), cc->sigma_ij.end(), sigma_ij);
    });
}

extern "C" mc_status mc_sample_range(const mc_tables *t, int h, int32_t unrooted_shape, int64_t node_lo,
                                     int64_t node_hi, uint64_t seed, uint64_t first_index, int64_t count,
                                     uint32_t *nodes, uint32_t *roots, int32_t *shapes, int32_t *classes,
                                     void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t, "tables is NULL");
        MC_REQUIRE(h >= 2 && h <= t->k, "h must be in 2..k");
        MC_REQUIRE(!t->level_missing(h), "level h was skipped (round skipping)");
        MC_REQUIRE(count >= 0, "count must be >= 0");
        refresh_tables(t, (cudaStream_t)stream);
        MC_REQUIRE(unrooted_shape < shape_catalog().n_unrooted[h], "unrooted shape out of range");
        if (count == 0) return;
        cudaStream_t s = (cudaStream_t)stream;
        const ClassCatalog *cc = class_catalog(h);
        Arena scratch(true);
        scratch.alloc = t->arena.alloc;
        scratch.stream = s;
        int *err = scratch.get<int>(2);
        MC_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
        SampleArgs a;
        fill_sample_args(a, t, h);
        RootIndex ri = root_index(t, h, unrooted_shape, scratch, err + 1, s, a.allow0, a.allow1, node_lo, node_hi);
        if (ri.R == 0) throw Error(MC_E_INVALID, "no colourful treelet of the requested size/shape");
        a.prefix = ri.prefix;
        a.R = ri.R;
        a.Xbase = ri.base;
        a.bucket = ri.bucket;
        a.D = ri.D;
        a.seed = seed;
        a.first_index = first_index;
        a.count = count;
        a.lut = cc->lut;
        a.nodes = nodes;
        a.roots = roots;
        a.shapes = shapes;
        a.classes = classes;
        a.hist = nullptr;
        a.ncls = (int)cc->codes.size();
        a.err = err;
        a.bytes = sample_byte_counter(scratch, s);
        a.next = batch_counter(scratch, s);
        launch_sampler(t, a, s);
        report_sample_bytes(a.bytes, s);
        int herr[2] = {0, 0};
        MC_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        if (herr[0] || herr[1]) throw Error(MC_E_INTERNAL, "sampler consistency check failed");
    });
}

// the star index of size h (built once per graph)
static u128 ensure_star_index(const mc_graph *gc, int h, cudaStream_t s)
{
    mc_graph *g = const_cast<mc_graph *>(gc);
    std::lock_guard<std::mutex> lock(g->star_mu);
    if (g->star_prefix[h]) return g->star_total[h];
    const int64_t n = g->n;
    Arena scratch(true);
    scratch.alloc = g->arena.alloc;
    scratch.stream = s;
    int *err = scratch.get<int>(1);
    MC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    u128 *p = g->arena.get<u128>((size_t)std::max<int64_t>(n, 1));
    const int64_t nb = bucket_count(n);
    uint32_t *bk = g->arena.get<uint32_t>((size_t)nb + 1);
    u128 *dD = scratch.get<u128>(1);
    u128 S = 0, D = 1;
    int herr = 0;
    if (n) {
        MC_LAUNCH("star_weights", s, star_weights_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->row_ptr, n, h - 1, p, err));
        inclusive_scan_u128(p, n, err, scratch, s);
        build_buckets(p, n, nb, dD, bk, s);
        MC_CUDA(cudaMemcpyAsync(&S, p + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(&D, dD, sizeof(u128), cudaMemcpyDeviceToHost, s));
    }
    MC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error(MC_E_OVERFLOW, "the number of stars does not fit in 128 bits");
    g->star_total[h] = S;
    g->star_D[h] = D;
    g->star_bucket[h] = bk;
    g->star_prefix[h] = p;  // published last
    return S;
}

// `count` stars from index first_index into the given outputs and/or a
// class histogram (device)
static void run_stars(const mc_graph *g, int h, uint64_t seed, uint64_t first_index, int64_t count,
                      uint32_t *nodes, uint32_t *centres, int32_t *classes, unsigned long long *hist,
                      Arena &scratch, cudaStream_t s)
{
    const u128 S = ensure_star_index(g, h, s);
    if (S == 0) throw Error(MC_E_INVALID, "the graph has no star of this size");
    const ClassCatalog *cc = class_catalog(h);
    int *err = scratch.get<int>(1);
    MC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    StarArgs a{};
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.prefix = g->star_prefix[h];
    a.bucket = g->star_bucket[h];
    a.D = g->star_D[h];
    a.n = g->n;
    a.S = S;
    a.h = h;
    a.seed = seed;
    a.first_index = first_index;
    a.count = count;
    a.lut = cc->lut;
    a.nodes = nodes;
    a.centres = centres;
    a.classes = classes;
    a.hist = hist;
    a.err = err;
    if ((S >> 64) == 0)
        MC_LAUNCH("star_sample", s, star_kernel<uint64_t><<<grid_for(count, 256), 256, 0, s>>>(a));
    else
        MC_LAUNCH("star_sample", s, star_kernel<u128><<<grid_for(count, 256), 256, 0, s>>>(a));
    int herr = 0;
    MC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error(MC_E_INTERNAL, "star sampler consistency check failed");
}

extern "C" mc_status mc_star_total(const mc_graph *g, int h, uint64_t total[2], void *stream)
{
    return guarded([&] {
        MC_REQUIRE(g && total, "NULL argument");
        MC_REQUIRE(h >= 2 && h <= MAXK, "h must be in 2..8");
        const u128 S = ensure_star_index(g, h, (cudaStream_t)stream);
        total[0] = (uint64_t)S;
        total[1] = (uint64_t)(S >> 64);
    });
}

extern "C" mc_status mc_sample_stars(const mc_graph *g, int h, uint64_t seed, uint64_t first_index, int64_t count,
                                     uint32_t *nodes, uint32_t *centres, int32_t *classes, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(g, "graph is NULL");
        MC_REQUIRE(h >= 2 && h <= MAXK, "h must be in 2..8");
        MC_REQUIRE(count >= 0, "count must be >= 0");
        if (count == 0) return;
        cudaStream_t s = (cudaStream_t)stream;
        Arena scratch(true);
        scratch.alloc = g->arena.alloc;
        scratch.stream = s;
        run_stars(g, h, seed, first_index, count, nodes, centres, classes, nullptr, scratch, s);
    });
}

extern "C" mc_status mc_sample(const mc_tables *t, int h, int32_t unrooted_shape, uint64_t seed,
                               uint64_t first_index, int64_t count, uint32_t *nodes, uint32_t *roots,
                               int32_t *shapes, int32_t *classes, void *stream)
{
    return mc_sample_range(t, h, unrooted_shape, 0, 0, seed, first_index, count, nodes, roots, shapes, classes,
                           stream);
}

// Round-skipped level k: sigma'_i = sum_j sigma_ij a_j (the counted
// spanning trees of H_i, each weighted by its rooted copies in the table)
// and sigma*_i (the spanning stars of H_i).
static void skip_sigmas(const mc_tables *t, const ClassCatalog *cc, int h, std::vector<int64_t> &sp,
                        std::vector<int64_t> &ss)
{
    const int ncls = (int)cc->codes.size(), nu = shape_catalog().n_unrooted[h];
    sp.assign((size_t)ncls, 0);
    ss.assign((size_t)ncls, 0);
    for (int i = 0; i < ncls; ++i)
        for (int j = 0; j < nu; ++j) {
            const int64_t sij = cc->sigma_ij[(size_t)i * nu + j];
            sp[(size_t)i] += sij * t->copies_k[j];
            if (t->copies_k[j] == 0) ss[(size_t)i] += sij;
        }
}

// The graphlets only stars span (sigma'_i = 0), from star_samples
// uncoloured stars: g_i = (S * hits*_i) / (sigma*_i * star_samples), their
// hits the star hits; 0 without stars or star samples.
static void star_estimates(const mc_tables *t, int h, const mc_estimate_params *p, const std::vector<int64_t> &sp,
                           const std::vector<int64_t> &ss, double *est, uint64_t *hits, Arena &scratch,
                           cudaStream_t s)
{
    const int ncls = (int)sp.size();
    std::vector<unsigned long long> sh((size_t)ncls, 0);
    const u128 S = ensure_star_index(t->g, h, s);
    if (S > 0 && p->star_samples > 0) {
        unsigned long long *dh = scratch.get<unsigned long long>((size_t)ncls);
        MC_CUDA(cudaMemsetAsync(dh, 0, (size_t)ncls * 8, s));
        run_stars(t->g, h, p->seed, p->first_index, p->star_samples, nullptr, nullptr, nullptr, dh, scratch, s);
        MC_CUDA(cudaMemcpyAsync(sh.data(), dh, (size_t)ncls * 8, cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
    }
    const double Sd = (double)S;
    for (int i = 0; i < ncls; ++i) {
        if (sp[(size_t)i] != 0) continue;
        hits[i] = sh[(size_t)i];
        est[i] = (S > 0 && p->star_samples > 0 && ss[(size_t)i] > 0)
                     ? (Sd * (double)sh[(size_t)i]) / ((double)ss[(size_t)i] * (double)p->star_samples)
                     : 0.0;
    }
}

extern "C" mc_status mc_estimate_counts(const mc_tables *t, const mc_estimate_params *p, double *est,
                                        uint64_t *hits, mc_estimate_stats *stats, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t && p && est && hits, "NULL argument");
        const int h = p->h;
        MC_REQUIRE(h >= 2 && h <= t->k, "h must be in 2..k");
        MC_REQUIRE(!t->level_missing(h), "level h was skipped (round skipping)");
        MC_REQUIRE(p->samples >= 0, "samples must be >= 0");
        refresh_tables(t, (cudaStream_t)stream);
        MC_REQUIRE(p->mode == MC_EST_UNIFORM || p->mode == MC_EST_AGS, "unknown mode");
        cudaStream_t s = (cudaStream_t)stream;
        const ClassCatalog *cc = class_catalog_sigma(h);
        const int ncls = (int)cc->codes.size();
        const ShapeCatalog &cat = shape_catalog();
        Arena scratch(true);
        scratch.alloc = t->arena.alloc;
        scratch.stream = s;
        int *err = scratch.get<int>(2);
        MC_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
        mc_estimate_stats st{};
        MC_REQUIRE((uint64_t)(t->k - 1) * p->colour_bias_q32 <= 4294967296ull, "(k-1) lambda must be at most 1");
        const double ip = inv_colourful_prob_biased(t->k, h, p->colour_bias_q32);
        // round-skipped level k: sigma' replaces sigma, R replaces t, and the
        // graphlets only stars span come from uncoloured stars
        const bool skipped = t->skip_round && h == t->k;
        std::vector<int64_t> sig_prime, sig_star;
        if (skipped) {
            skip_sigmas(t, cc, h, sig_prime, sig_star);
            MC_REQUIRE(p->star_samples >= 0, "star_samples must be >= 0");
            MC_REQUIRE(p->star_samples == 0 || (p->node_lo <= 0 && (p->node_hi <= 0 || p->node_hi == t->g->n)),
                       "star samples cover the whole graph: no node range with star_samples");
        }
        if (p->mode == MC_EST_UNIFORM) {
            MC_REQUIRE(p->samples > 0, "uniform estimation needs samples > 0");
            unsigned long long *dh = scratch.get<unsigned long long>((size_t)ncls);
            int64_t *dsig = scratch.get<int64_t>((size_t)ncls);
            double *dest = scratch.get<double>((size_t)ncls);
            MC_CUDA(cudaMemsetAsync(dh, 0, (size_t)ncls * 8, s));
            MC_CUDA(cudaMemcpyAsync(dsig, skipped ? sig_prime.data() : cc->sigma_i.data(), (size_t)ncls * 8,
                                    cudaMemcpyHostToDevice, s));
            SampleArgs a;
            fill_sample_args(a, t, h);
            RootIndex ri = root_index(t, h, -1, scratch, err + 1, s, a.allow0, a.allow1, p->node_lo, p->node_hi);
            if (ri.R == 0) throw Error(MC_E_INVALID, "no colourful treelet of size h");
            a.prefix = ri.prefix;
            a.R = ri.R;
            a.Xbase = ri.base;
            a.bucket = ri.bucket;
            a.D = ri.D;
            a.seed = p->seed;
            a.first_index = p->first_index;
            a.count = p->samples;
            a.lut = cc->lut;
            a.hist = dh;
            a.ncls = ncls;
            a.err = err;
            a.bytes = sample_byte_counter(scratch, s);
            a.next = batch_counter(scratch, s);
            launch_sampler(t, a, s);
            report_sample_bytes(a.bytes, s);
            const u128 tnum = skipped ? ri.R : ri.R / (u128)t->copies_div(h);
            MC_LAUNCH("estimate", s, uniform_estimate_kernel<<<(ncls + 127) / 128, 128, 0, s>>>(dh, dsig, ncls, tnum, p->samples, ip, dest));
            std::vector<unsigned long long> hh((size_t)ncls);
            MC_CUDA(cudaMemcpyAsync(hh.data(), dh, (size_t)ncls * 8, cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(est, dest, (size_t)ncls * 8, cudaMemcpyDeviceToHost, s));
            int herr[2] = {0, 0};
            MC_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaStreamSynchronize(s));
            if (herr[0] || herr[1]) throw Error(MC_E_INTERNAL, "sampler consistency check failed");
            for (int i = 0; i < ncls; ++i) hits[i] = hh[i];
            st.samples = p->samples;
            st.batches = 1;
            if (skipped) star_estimates(t, h, p, sig_prime, sig_star, est, hits, scratch, s);
        } else {
            // Algorithm AGS.  Every treelet T_j has its own stream of sample
            // indices (the n-th sample drawn with T_j has index first_index +
            // j * 2^40 + n), so samples can be drawn ahead: a launch draws a
            // run for the current treelet and a short run for every other
            // treelet whose queue is empty, and the host replays the
            // algorithm one sample at a time, taking each from the queue of
            // the treelet it has chosen.  One launch stays in flight while
            // the host replays, so drawing and replaying overlap.  The
            // outcome is the one of drawing one sample at a time; what is
            // left in the queues at the end was drawn ahead and not used.
            int64_t cbar = p->cbar;
            if (cbar <= 0) {
                MC_REQUIRE(p->eps > 0 && p->delta > 0 && p->delta < 1, "AGS needs cbar or (eps, delta)");
                cbar = (int64_t)std::ceil(4.0 / (p->eps * p->eps) * std::log(2.0 * ncls / p->delta));
            }
            MC_REQUIRE(p->samples <= ((int64_t)1 << 40), "AGS draws at most 2^40 samples");
            const int nu = cat.n_unrooted[h];
            std::vector<u128> tj(nu);
            std::vector<double> tjd(nu);
            std::vector<std::pair<uint64_t, uint64_t>> allows;
            // every treelet's root index once: its rooted total gives t_j
            const std::vector<RootIndex> ris =
                treelet_root_indexes(t, h, scratch, err + 1, s, allows, p->node_lo, p->node_hi);
            for (int j = 0; j < nu; ++j) {
                tj[j] = unrooted_from_rooted(t, h, j, ris[j].R);
                tjd[j] = (double)tj[j];
            }
            int cur = -1;
            for (int j = 0; j < nu; ++j)
                if (tj[j] > 0 && (cur < 0 || tj[j] > tj[cur])) cur = j;
            std::vector<int64_t> nj(nu, 0);
            std::vector<uint64_t> hv((size_t)ncls, 0);
            std::vector<double> w((size_t)ncls, 0.0);
            std::vector<uint8_t> covered((size_t)ncls, 0);
            int64_t drawn = 0, ncov = 0;
            // run lengths: the current treelet's first run, its largest, and
            // the short run drawn ahead for the others
            const int64_t bmin = p->batch > 0 ? p->batch : 65536;
            const int64_t bmax = p->batch > 0 ? p->batch : (int64_t)1 << 22;
            const int64_t ahead = std::min<int64_t>(bmax, 4096);
            const int64_t cap = bmax + (int64_t)nu * ahead;  // samples of one launch, at most
            int32_t *dcls = scratch.get<int32_t>((size_t)cap);
            SampleSeg *dseg = scratch.get<SampleSeg>((size_t)nu);
            // the part table, then the class ids of one launch
            const size_t seg_bytes = ((size_t)nu * sizeof(SampleSeg) + 255) & ~(size_t)255;
            char *pin = (char *)pinned_scratch(seg_bytes + (size_t)cap * sizeof(int32_t));
            SampleSeg *hseg = (SampleSeg *)pin;
            int32_t *hcls = (int32_t *)(pin + seg_bytes);
            EventHandle done;
            std::vector<std::vector<int32_t>> queue((size_t)nu);  // drawn, not yet used, in index order
            std::vector<size_t> qpos((size_t)nu, 0);
            std::vector<int64_t> queued(nu, 0);  // samples drawn with T_j
            std::vector<int64_t> amount(nu, 0);                // the launch in flight, per treelet
            int streak = 0;  // launches since the current treelet was chosen
            bool in_flight = false;
            unsigned long long *bytes = nullptr;
            struct Drain {  // an error leaves no copy running into the buffers above
                const bool &f;
                cudaEvent_t e;
                ~Drain() { if (f) cudaEventSynchronize(e); }
            } drain{in_flight, done.e};
            std::vector<int> cov_list;  // covered graphlets, ascending
            auto weight = [&](int i) {
                double acc = 0.0;
                for (int j = 0; j < nu; ++j)
                    if (tj[j] > 0) acc += (double)(nj[j] * cc->sigma_ij[(size_t)i * nu + j]) / tjd[j];
                w[(size_t)i] = acc;
            };
            auto weights = [&] {
                for (int i = 0; i < ncls; ++i) weight(i);
            };
            // Run lengths only (the outcome does not depend on them): hits per
            // class among the samples used from each T_j predict how many more
            // T_j needs until some graphlet is covered.
            std::vector<uint64_t> hj((size_t)nu * ncls, 0);
            auto predict = [&](int j) -> int64_t {
                if (nj[j] == 0) return -1;
                double best = -1.0;
                for (int i = 0; i < ncls; ++i) {
                    const uint64_t c = hj[(size_t)j * ncls + i];
                    if (covered[(size_t)i] || c == 0) continue;
                    const double need = (double)(cbar - (int64_t)hv[(size_t)i]) * (double)nj[j] / (double)c;
                    if (best < 0.0 || need < best) best = need;
                }
                return best < 0.0 ? -1 : (int64_t)best;
            };
            auto left = [&](int j) { return (int64_t)(queue[j].size() - qpos[j]); };
            // plan and launch the next draw (nothing if nothing is wanted)
            auto issue = [&] {
                int64_t total = 0;
                for (int j = 0; j < nu; ++j) {
                    amount[j] = 0;
                    if (tj[j] == 0) continue;
                    const int64_t budget = p->samples - drawn - left(j);  // what T_j could still use
                    if (budget <= 0) continue;
                    if (j == cur) {
                        int64_t want = bmin;
                        if (p->batch <= 0) {
                            const int64_t q = predict(j) - left(j);
                            if (q >= 0) want = std::max<int64_t>(want, q + q / 4 + 4096);
                            // runs double while the treelet stays chosen
                            want = std::max(want, bmin << std::min(streak, 6));
                        }
                        amount[j] = std::min(std::min(want, bmax), budget);
                    } else if (left(j) == 0) {
                        amount[j] = std::min(ahead, budget);
                    }
                    total += amount[j];
                }
                if (total == 0) return;
                SampleArgs a;
                fill_sample_args(a, t, h);
                int nseg = 0;
                int64_t end = 0;
                for (int j = 0; j < nu; ++j) {
                    if (amount[j] == 0) continue;
                    SampleSeg &sg = hseg[nseg++];
                    end += amount[j];
                    sg.end = end;
                    sg.first_index = p->first_index + ((uint64_t)j << 40) + (uint64_t)queued[j];
                    sg.prefix = ris[j].prefix;
                    sg.bucket = ris[j].bucket;
                    sg.R = ris[j].R;
                    sg.Xbase = ris[j].base;
                    sg.D = ris[j].D;
                    sg.allow0 = allows[j].first;
                    sg.allow1 = allows[j].second;
                    queued[j] += amount[j];
                    if (ris[j].R + ris[j].base > a.R + a.Xbase) { a.R = ris[j].R; a.Xbase = ris[j].base; }  // width test
                }
                MC_CUDA(cudaMemcpyAsync(dseg, hseg, (size_t)nseg * sizeof(SampleSeg), cudaMemcpyHostToDevice, s));
                a.seg = dseg;
                a.nseg = nseg;
                a.seed = p->seed;
                a.count = total;
                a.lut = cc->lut;
                a.classes = dcls;
                a.ncls = ncls;
                a.err = err;
                a.bytes = bytes = sample_byte_counter(scratch, s);
                a.next = batch_counter(scratch, s);
                launch_sampler(t, a, s);
                MC_CUDA(cudaMemcpyAsync(hcls, dcls, (size_t)total * 4, cudaMemcpyDeviceToHost, s));
                MC_CUDA(cudaEventRecord(done.e, s));
                in_flight = true;
                st.batches++;
            };
            // wait for the launch in flight and append its samples to the queues
            auto collect = [&] {
                MC_CUDA(cudaEventSynchronize(done.e));
                report_sample_bytes(bytes, s);
                int64_t off = 0;
                for (int j = 0; j < nu; ++j) {
                    if (amount[j] == 0) continue;
                    std::vector<int32_t> &qj = queue[j];
                    qj.erase(qj.begin(), qj.begin() + (std::ptrdiff_t)qpos[j]);
                    qpos[j] = 0;
                    qj.insert(qj.end(), hcls + off, hcls + off + amount[j]);
                    off += amount[j];
                    amount[j] = 0;
                }
                in_flight = false;
            };
            int64_t target = ncls;  // round-skipped: the graphlets only stars span are left to the stars
            if (skipped) {
                target = 0;
                for (int i = 0; i < ncls; ++i) target += sig_prime[(size_t)i] > 0;
            }
            while (cur >= 0 && ncov < target && drawn < p->samples) {
                if (left(cur) == 0) {
                    if (in_flight) collect();
                    if (left(cur) == 0) {  // the launch in flight had nothing for T_j
                        issue();
                        collect();
                    }
                    issue();  // the next draw runs while the host replays
                    ++streak;
                }
                // replay until the queue runs dry, the budget ends or a
                // graphlet becomes covered
                const int32_t *qd = queue[cur].data();
                const size_t q0 = qpos[cur];
                const size_t qe = q0 + (size_t)std::min<int64_t>(left(cur), p->samples - drawn);
                uint64_t *hjc = &hj[(size_t)cur * ncls];
                size_t q = q0;
                int hit = -1;
                while (q < qe) {
                    const int32_t i = qd[q++];
                    if ((uint32_t)i >= (uint32_t)ncls) throw Error(MC_E_INTERNAL, "AGS: bad class id");
                    hjc[i]++;
                    if (++hv[(size_t)i] == (uint64_t)cbar && !covered[(size_t)i]) { hit = i; break; }
                }
                nj[cur] += (int64_t)(q - q0);
                drawn += (int64_t)(q - q0);
                qpos[cur] = q;
                if (hit >= 0) {
                    covered[(size_t)hit] = 1;
                    cov_list.insert(std::lower_bound(cov_list.begin(), cov_list.end(), hit), hit);
                    ncov++;
                    st.switches++;
                    // the choice reads w_i of the covered graphlets only: the
                    // same sums, in the same order, over the covered list
                    // (ascending) instead of every class
                    for (const int i : cov_list) weight(i);
                    int best = -1;
                    double bestv = 0.0;
                    for (int j = 0; j < nu; ++j) {
                        if (tj[j] == 0) continue;
                        double acc = 0.0;
                        for (const int a2 : cov_list)
                            acc += ((double)cc->sigma_ij[(size_t)a2 * nu + j] * (double)hv[(size_t)a2]) / w[(size_t)a2];
                        const double val = acc / tjd[j];
                        if (best < 0 || val < bestv) { best = j; bestv = val; }
                    }
                    if (best != cur) streak = 0;
                    cur = best;
                }
            }
            if (in_flight) collect();
            for (int j = 0; j < nu; ++j) st.discarded += left(j);
            weights();
            for (int i = 0; i < ncls; ++i) {
                hits[i] = hv[(size_t)i];
                est[i] = w[(size_t)i] > 0.0 ? ((double)hv[(size_t)i] / w[(size_t)i]) * ip : 0.0;
            }
            int herr[2] = {0, 0};
            MC_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaStreamSynchronize(s));
            if (herr[0] || herr[1]) throw Error(MC_E_INTERNAL, "sampler consistency check failed");
            st.samples = drawn;
            st.covered = ncov;
            if (skipped) star_estimates(t, h, p, sig_prime, sig_star, est, hits, scratch, s);
        }
        if (stats) *stats = st;
    });
}

// ---------------------------------------------------------------------------
// Uniform estimation without device allocation: the scratch of
// mc_estimate_counts' uniform mode (histogram, sigma, estimates, error
// flags) lives in one static device array instead of allocator memory.
// ---------------------------------------------------------------------------
namespace mc {

constexpr int NOALLOC_MAX_CLASSES = 12288;  // >= 11117, the connected 8-node graphs

struct NoAllocScratch {
    unsigned long long hist[NOALLOC_MAX_CLASSES];
    int64_t sigma[NOALLOC_MAX_CLASSES];
    double est[NOALLOC_MAX_CLASSES];
    int err[4];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

static std::mutex g_noalloc_mutex;
static std::map<int, NoAllocScratch *> g_noalloc_addr;

// Device address of the static scratch on the current device, looked up
// once per device (host code cannot use the symbol itself as a pointer).
static NoAllocScratch *noalloc_scratch()
{
    int dev = 0;
    MC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) return it->second;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        throw Error(MC_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = (NoAllocScratch *)p;
    return (NoAllocScratch *)p;
}

// The class catalogue of size h if it already exists with sigma, else NULL
// (never builds it: that would allocate).
static const ClassCatalog *existing_catalogue(int h)
{
    int dev = 0;
    MC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_cls_mutex);
    auto it = g_cls.find(std::make_pair(dev, h));
    if (it == g_cls.end() || !it->second->sigma_ready) return nullptr;
    return it->second;
}

}  // namespace mc

extern "C" mc_status mc_estimate_uniform_noalloc(const mc_tables *t, int h, uint64_t seed, uint64_t first_index,
                                                 int64_t samples, double *est, uint64_t *hits, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(t && est && hits, "NULL argument");
        MC_REQUIRE(h >= 2 && h <= t->k, "h must be in 2..k");
        MC_REQUIRE(!(t->skip_round && h >= t->k - 1), "not available on round-skipped levels");
        MC_REQUIRE(samples > 0, "samples must be > 0");
        const ClassCatalog *cc = existing_catalogue(h);
        if (!cc)
            throw Error(MC_E_INVALID, "the graphlet catalogue of this size does not exist on this device yet "
                                      "(creating it allocates); call mc_sigma(h) first");
        const int ncls = (int)cc->codes.size();
        if (ncls > NOALLOC_MAX_CLASSES)
            throw Error(MC_E_UNSUPPORTED, "more graphlet classes than the static scratch holds (" +
                                              std::to_string(NOALLOC_MAX_CLASSES) + ")");
        // the level's root index, read under the lock that guards its
        // publication; one made for an older colouring is refused, since
        // remaking it allocates
        const u128 *prefix = nullptr;
        const uint32_t *bucket = nullptr;
        u128 R = 0, D = 1;
        {
            std::lock_guard<std::mutex> lock(const_cast<mc_tables *>(t)->idx_mu);
            MC_REQUIRE(!t->stale && t->broken.empty(),
                       "tables rebuilt since their totals were read: call mc_tables_status first");
            if (!t->prefix[h])
                throw Error(MC_E_INVALID, "the root index of this level does not exist yet (creating it "
                                          "allocates); call mc_total(h) first");
            if (t->level_stale[h])
                throw Error(MC_E_INVALID, "the root index of this level predates the last rebuild (remaking it "
                                          "allocates); call mc_total(h) first");
            prefix = t->prefix[h];
            bucket = t->bucket[h];
            R = t->R[h];
            D = t->bucketD[h];
        }
        if (R == 0) throw Error(MC_E_INVALID, "no colourful treelet of size h");
        cudaStream_t s = (cudaStream_t)stream;
        NoAllocScratch *scr = noalloc_scratch();
        MC_CUDA(cudaMemsetAsync(scr->hist, 0, (size_t)ncls * sizeof(unsigned long long), s));
        MC_CUDA(cudaMemsetAsync(scr->err, 0, sizeof(scr->err), s));
        MC_CUDA(cudaMemcpyAsync(scr->sigma, cc->sigma_i.data(), (size_t)ncls * sizeof(int64_t),
                                cudaMemcpyHostToDevice, s));
        SampleArgs a;
        fill_sample_args(a, t, h);
        const ShapeCatalog &cat = shape_catalog();
        a.allow0 = a.allow1 = 0;
        for (int i = 0; i < cat.r[h]; ++i) {
            if (i < 64) a.allow0 |= 1ull << i; else a.allow1 |= 1ull << (i - 64);
        }
        a.prefix = prefix;
        a.R = R;
        a.bucket = bucket;
        a.D = D;
        a.seed = seed;
        a.first_index = first_index;
        a.count = samples;
        a.lut = cc->lut;
        a.hist = scr->hist;
        a.ncls = ncls;
        a.err = scr->err;
        launch_sampler(t, a, s);
        const double ip = inv_colourful_prob(t->k, h);
        MC_LAUNCH("estimate", s, uniform_estimate_kernel<<<(ncls + 127) / 128, 128, 0, s>>>(
                                     scr->hist, scr->sigma, ncls, R / (u128)t->copies_div(h), samples, ip, scr->est));
        int herr[2] = {0, 0};
        MC_CUDA(cudaMemcpyAsync(hits, scr->hist, (size_t)ncls * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(est, scr->est, (size_t)ncls * sizeof(double), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(herr, scr->err, sizeof(herr), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        if (herr[0] || herr[1]) throw Error(MC_E_INTERNAL, "sampler consistency check failed");
    });
}
