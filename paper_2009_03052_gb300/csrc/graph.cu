// graph.cu -- error plumbing, device memory, graph loading and validation,
// colouring (Section 2.1).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace mc {

void inclusive_scan_u128(u128 *x, int64_t n, int *err, Arena &scratch, cudaStream_t s);

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

void *Allocator::alloc(size_t bytes, cudaStream_t s) const
{
    if (custom) return a.alloc(bytes, a.ctx, (void *)s);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Allocator::release(void *p, size_t bytes, cudaStream_t s) const
{
    if (!p) return;
    if (custom) a.free(p, bytes, a.ctx, (void *)s);
    else cudaFree(p);
}

void Arena::release(void *p)
{
    for (size_t i = 0; i < blocks.size(); ++i)
        if (blocks[i].first == p) {
            if (scratch && !alloc.custom) cudaFreeAsync(p, stream);
            else alloc.release(p, blocks[i].second, stream);
            blocks.erase(blocks.begin() + (long)i);
            return;
        }
}

void Arena::release_all()
{
    for (auto &b : blocks) {
        if (scratch && !alloc.custom) cudaFreeAsync(b.first, stream);
        else alloc.release(b.first, b.second, stream);
    }
    blocks.clear();
}

// ---------------------------------------------------------------------------
// validation (offsets already checked on the host): one thread per directed
// edge (u, col[e]); flags: bit 0 out of range, bit 1 self-loop, bit 2 not
// strictly ascending, bit 3 not symmetric.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t row_of(const int64_t *row_ptr, int64_t n, int64_t e)
{
    int64_t lo = 0, hi = n;  // last node with row_ptr[node] <= e
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void validate_edges(const int64_t *row_ptr, const uint32_t *col, int64_t n, int64_t nnz,
                               int *flags)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = row_of(row_ptr, n, e);
        const uint32_t w = col[e];
        if (w >= n) { atomicOr(flags, 1); continue; }
        if (w == u) atomicOr(flags, 2);
        if (e > row_ptr[u] && col[e - 1] >= w) atomicOr(flags, 4);
        int64_t lo = row_ptr[w], hi = row_ptr[w + 1];
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (col[mid] < (uint32_t)u) lo = mid + 1; else hi = mid;
        }
        if (lo >= row_ptr[w + 1] || col[lo] != (uint32_t)u) atomicOr(flags, 8);
    }
}

__global__ void validate_offsets(const int64_t *row_ptr, int64_t n, int64_t nnz, int *flags)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (v == 0 && row_ptr[0] != 0) atomicOr(flags, 16);
        if (v == n && row_ptr[n] != nnz) atomicOr(flags, 16);
        if (v < n && row_ptr[v] > row_ptr[v + 1]) atomicOr(flags, 16);
    }
}

// per node: number of hub chunks (0 unless degree > HUB_CHUNK) and whether
// it is a hub; the largest degree
__global__ void degree_stats(const int64_t *row_ptr, int64_t n, u128 *nch, u128 *nhub, unsigned long long *maxdeg)
{
    unsigned long long md = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        nch[v] = d > HUB_CHUNK ? (u128)((d + HUB_CHUNK - 1) / HUB_CHUNK) : (u128)0;
        nhub[v] = d > HUB_CHUNK ? 1 : 0;
        if ((unsigned long long)d > md) md = (unsigned long long)d;
    }
    // one atomic per warp, not per thread (a single address serialises them)
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, md, o);
        if (x > md) md = x;
    }
    if ((threadIdx.x & 31) == 0 && md) atomicMax(maxdeg, md);
}

// from the inclusive prefixes of chunk and hub counts: every hub writes its
// chunks (node, first edge, end edge), its entry in the hub list and its
// first chunk
__global__ void hub_chunks(const int64_t *row_ptr, int64_t n, const u128 *nch, const u128 *nhub,
                           uint32_t *chunk_node, int64_t *chunk_e0, int64_t *chunk_e1, uint32_t *hub_node,
                           int64_t *hub_chunk0, int32_t *node_chunk0, int64_t n_hubs, int64_t n_chunks)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c1 = (int64_t)nch[v], c0 = v ? (int64_t)nch[v - 1] : 0;
        if (c1 == c0) { node_chunk0[v] = -1; continue; }
        const int64_t hid = (int64_t)nhub[v] - 1;
        hub_node[hid] = (uint32_t)v;
        hub_chunk0[hid] = c0;
        if (hid == n_hubs - 1) hub_chunk0[n_hubs] = n_chunks;
        node_chunk0[v] = (int32_t)c0;
        const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        for (int64_t c = c0; c < c1; ++c) {
            chunk_node[c] = (uint32_t)v;
            chunk_e0[c] = e0 + (c - c0) * HUB_CHUNK;
            chunk_e1[c] = min(e1, e0 + (c - c0 + 1) * HUB_CHUNK);
        }
    }
    if (n_hubs == 0 && blockIdx.x == 0 && threadIdx.x == 0) hub_chunk0[0] = 0;
}

// Nodes of degree <= HUB_CHUNK by degree: a histogram of the degrees, then
// each node takes the next slot of its degree's range (ranges in descending
// order of degree; the order inside a range does not matter).
__global__ void degree_hist_kernel(const int64_t *__restrict__ row_ptr, int64_t n, unsigned *hist)
{
    __shared__ unsigned sh[HUB_CHUNK + 1];
    for (int i = threadIdx.x; i <= HUB_CHUNK; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d <= HUB_CHUNK) atomicAdd(&sh[d], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= HUB_CHUNK; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// A block takes a tile of blockDim nodes at a time: shared-memory counts
// give each node its place among the tile's nodes of its degree, one global
// atomic per degree present reserves the tile's run in that degree's
// bucket.  (The order inside a bucket is free: the sums are per node.)
__global__ void degree_order_kernel(const int64_t *__restrict__ row_ptr, int64_t n, unsigned *cursor,
                                    uint4 *__restrict__ sched)
{
    __shared__ unsigned cnt[HUB_CHUNK + 1], base[HUB_CHUNK + 1];
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < n; t0 += (int64_t)gridDim.x * blockDim.x) {
        for (int i = threadIdx.x; i <= HUB_CHUNK; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const int64_t v = t0 + threadIdx.x;
        int64_t e0 = 0, d = HUB_CHUNK + 1;
        if (v < n) {
            e0 = row_ptr[v];
            d = row_ptr[v + 1] - e0;
        }
        unsigned local = 0;
        if (d <= HUB_CHUNK) local = atomicAdd(&cnt[d], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i <= HUB_CHUNK; i += blockDim.x)
            base[i] = cnt[i] ? atomicAdd(&cursor[i], cnt[i]) : 0u;
        __syncthreads();
        if (d <= HUB_CHUNK)
            sched[base[d] + local] =
                make_uint4((uint32_t)v, (uint32_t)e0, (uint32_t)((uint64_t)e0 >> 32), (uint32_t)d);
        __syncthreads();  // cnt and base are reused by the next tile
    }
}

// Hubs of more than HUB_SERIAL chunks (their chunk sums get a warp each).
__global__ void big_hubs_kernel(const int64_t *__restrict__ hub_chunk0, int64_t n_hubs, unsigned *count,
                                uint32_t *__restrict__ big)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_hubs;
         i += (int64_t)gridDim.x * blockDim.x)
        if (hub_chunk0[i + 1] - hub_chunk0[i] > HUB_SERIAL) big[atomicAdd(count, 1u)] = (uint32_t)i;
}

// Colouring: c_v = floor(k * x0 / 2^32), x0 the first Philox4x32-10 word at
// counter (v, 0, 0, 0xC010) and key = seed.
__global__ void color_kernel(int64_t n, int k, uint64_t seed, uint8_t *colors)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)v, 0u, 0u, 0xC010u};
        philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        colors[v] = (uint8_t)(((uint64_t)c[0] * (uint64_t)k) >> 32);
    }
}

// Biased colouring (Section 3.5): the same Philox word; colour 1 + x / L
// when x < (k-1) L, else 0 (probability L / 2^32 for each of colours 1..k-1).
__global__ void color_biased_kernel(int64_t n, int k, uint64_t seed, uint32_t L, uint8_t *colors)
{
    const uint64_t rare = (uint64_t)(k - 1) * L;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)v, 0u, 0u, 0xC010u};
        philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        colors[v] = (uint8_t)((uint64_t)c[0] < rare ? 1u + c[0] / L : 0u);
    }
}

// ---------------------------------------------------------------------------
// tracing
// ---------------------------------------------------------------------------
namespace {
struct ProfState {
    std::mutex mu;
    bool on = false;     // time every launch
    bool count = false;  // the sampler counts its bytes (an instantiation of its own)
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int64_t> launches;
    std::vector<int64_t> bytes;
    std::vector<std::pair<ProfSpan, int>> pending;
    std::vector<cudaEvent_t> pool;
};
ProfState &prof()
{
    static ProfState p;
    return p;
}
std::atomic<int64_t> g_launches{0};

cudaEvent_t take_event(ProfState &p)
{
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void drain(ProfState &p)
{
    for (auto &pe : p.pending) {
        float t = 0.f;
        if (cudaEventSynchronize(pe.first.b) == cudaSuccess &&
            cudaEventElapsedTime(&t, pe.first.a, pe.first.b) == cudaSuccess)
            p.ms[pe.second] += t;
        p.pool.push_back(pe.first.a);
        p.pool.push_back(pe.first.b);
    }
    p.pending.clear();
}
}  // namespace

ProfSpan prof_begin(const char *name, cudaStream_t s)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ProfSpan span;
    ProfState &p = prof();
    if (!p.on) return span;
    std::lock_guard<std::mutex> lock(p.mu);
    int id = -1;
    for (size_t i = 0; i < p.names.size(); ++i)
        if (p.names[i] == name) { id = (int)i; break; }
    if (id < 0) {
        id = (int)p.names.size();
        p.names.push_back(name);
        p.ms.push_back(0.0);
        p.launches.push_back(0);
        p.bytes.push_back(0);
    }
    span.id = id;
    span.a = take_event(p);
    span.b = take_event(p);
    if (span.a) cudaEventRecord(span.a, s);
    return span;
}

void prof_end(ProfSpan &span, cudaStream_t s)
{
    if (span.id < 0 || !span.a || !span.b) return;
    ProfState &p = prof();
    std::lock_guard<std::mutex> lock(p.mu);
    cudaEventRecord(span.b, s);
    p.launches[span.id]++;
    p.pending.emplace_back(span, span.id);
    if (p.pending.size() > 4096) drain(p);
}

bool prof_enabled() { return prof().on; }
bool prof_counting() { return prof().on && prof().count; }

void prof_add_bytes(const char *name, int64_t bytes)
{
    ProfState &p = prof();
    std::lock_guard<std::mutex> lock(p.mu);
    for (size_t i = 0; i < p.names.size(); ++i)
        if (p.names[i] == name) { p.bytes[i] += bytes; return; }
    p.names.push_back(name);
    p.ms.push_back(0.0);
    p.launches.push_back(0);
    p.bytes.push_back(bytes);
}

int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int grid_for(int64_t work, int block)
{
    int64_t g = (work + block - 1) / block;
    const int64_t cap = (int64_t)sm_count() * 32;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace mc

using namespace mc;

extern "C" const char *mc_last_error(void) { return g_last_error.c_str(); }

extern "C" mc_status mc_profile_enable(int on)
{
    return guarded([&] {
        ProfState &p = prof();
        std::lock_guard<std::mutex> lock(p.mu);
        p.on = on != 0;
        p.count = (on & 2) != 0;
    });
}

extern "C" mc_status mc_profile_reset(void)
{
    return guarded([&] {
        ProfState &p = prof();
        std::lock_guard<std::mutex> lock(p.mu);
        drain(p);
        std::fill(p.ms.begin(), p.ms.end(), 0.0);
        std::fill(p.launches.begin(), p.launches.end(), 0);
        std::fill(p.bytes.begin(), p.bytes.end(), 0);
    });
}

extern "C" mc_status mc_profile_read(char *names, size_t names_bytes, double *ms, int64_t *launches,
                                     int64_t *bytes, int max, int *count)
{
    return guarded([&] {
        ProfState &p = prof();
        std::lock_guard<std::mutex> lock(p.mu);
        drain(p);
        size_t pos = 0;
        int c = 0;
        for (size_t i = 0; i < p.names.size() && c < max; ++i) {
            const std::string &nm = p.names[i];
            if (names) {
                if (pos + nm.size() + 1 > names_bytes) break;
                std::memcpy(names + pos, nm.c_str(), nm.size() + 1);
                pos += nm.size() + 1;
            }
            if (ms) ms[c] = p.ms[i];
            if (launches) launches[c] = p.launches[i];
            if (bytes) bytes[c] = p.bytes[i];
            ++c;
        }
        if (count) *count = c;
    });
}

extern "C" int64_t mc_launch_count(void) { return g_launches.load(); }

extern "C" mc_status mc_load_graph(int64_t n, int64_t nnz, const int64_t *row_ptr, const uint32_t *col,
                                   uint32_t flags, const mc_allocator *alloc, void *stream,
                                   mc_graph **out)
{
    if (out) *out = nullptr;
    mc_graph *g = nullptr;
    mc_status st = guarded([&] {
        MC_REQUIRE(out, "out is NULL");
        MC_REQUIRE(n >= 0 && n < (int64_t)0xffffffffLL, "n must be in [0, 2^32 - 1)");
        MC_REQUIRE(nnz >= 0, "nnz must be >= 0");
        MC_REQUIRE(row_ptr && (col || nnz == 0), "row_ptr/col is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        g = new mc_graph();
        g->arena.stream = s;
        if (alloc) { g->arena.alloc.a = *alloc; g->arena.alloc.custom = true; }
        g->n = n;
        g->nnz = nnz;
        const bool on_dev = flags & MC_GRAPH_DEVICE_PTRS;
        const bool trusted = flags & MC_GRAPH_TRUSTED;
        const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        Arena scratch(true);
        scratch.alloc = g->arena.alloc;
        scratch.stream = s;
        int64_t *dstat = scratch.get<int64_t>(4);  // flags, max degree, #chunks, #hubs
        MC_CUDA(cudaMemsetAsync(dstat, 0, 4 * sizeof(int64_t), s));
        g->row_ptr = g->arena.get<int64_t>((size_t)n + 1);
        g->col = g->arena.get<uint32_t>((size_t)(nnz > 0 ? nnz : 1));
        MC_CUDA(cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int64_t) * (n + 1), kind, s));
        // A trusted graph's ids are copied on a side stream while the
        // degree statistics, hub chunks and schedule (which read only the
        // offsets) run on s; s joins the copy before the load returns, and
        // a failing load waits for it before its buffers are freed.
        struct SideCopy {
            cudaStream_t s2 = nullptr;
            cudaEvent_t ready = nullptr, done = nullptr;
            ~SideCopy()
            {
                if (s2) {
                    cudaStreamSynchronize(s2);
                    cudaStreamDestroy(s2);
                }
                if (ready) cudaEventDestroy(ready);
                if (done) cudaEventDestroy(done);
            }
        } side;
        if (nnz && trusted) {
            MC_CUDA(cudaStreamCreateWithFlags(&side.s2, cudaStreamNonBlocking));
            MC_CUDA(cudaEventCreateWithFlags(&side.ready, cudaEventDisableTiming));
            MC_CUDA(cudaEventCreateWithFlags(&side.done, cudaEventDisableTiming));
            MC_CUDA(cudaEventRecord(side.ready, s));  // after the allocations and the caller's work on s
            MC_CUDA(cudaStreamWaitEvent(side.s2, side.ready, 0));
            MC_CUDA(cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * nnz, kind, side.s2));
            MC_CUDA(cudaEventRecord(side.done, side.s2));
        } else if (nnz) {
            MC_CUDA(cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * nnz, kind, s));
        }
        // the offsets are checked before any kernel indexes with them: on the
        // host for host input, by a kernel (and a read-back) for device input
        if (!trusted) {
            if (!on_dev) {
                MC_REQUIRE(row_ptr[0] == 0 && row_ptr[n] == nnz, "row_ptr[0] must be 0 and row_ptr[n] must be nnz");
                for (int64_t v = 0; v < n; ++v)
                    MC_REQUIRE(row_ptr[v] <= row_ptr[v + 1], "row_ptr must be non-decreasing");
            } else {
                MC_LAUNCH("validate_offsets", s, validate_offsets<<<grid_for(n + 1, 256), 256, 0, s>>>(
                                                     g->row_ptr, n, nnz, (int *)dstat));
                int hf = 0;
                MC_CUDA(cudaMemcpyAsync(&hf, dstat, sizeof(int), cudaMemcpyDeviceToHost, s));
                MC_CUDA(cudaStreamSynchronize(s));
                MC_REQUIRE(hf == 0, "row_ptr must start at 0, end at nnz and be non-decreasing");
            }
            if (n > 0 && nnz)
                MC_LAUNCH("validate_edges", s, validate_edges<<<grid_for(nnz, 256), 256, 0, s>>>(
                                                   g->row_ptr, g->col, n, nnz, (int *)dstat));
        }
        // hub chunks, built on the device: chunk counts per node, their
        // prefix, then one thread per hub writes its chunks
        u128 *nch = scratch.get<u128>((size_t)(n > 0 ? n : 1));
        u128 *nhub = scratch.get<u128>((size_t)(n > 0 ? n : 1));
        int *serr = scratch.get<int>(1);
        MC_CUDA(cudaMemsetAsync(serr, 0, sizeof(int), s));
        if (n > 0) {
            MC_LAUNCH("degree_stats", s, degree_stats<<<grid_for(n, 256), 256, 0, s>>>(
                                             g->row_ptr, n, nch, nhub, (unsigned long long *)(dstat + 1)));
            inclusive_scan_u128(nch, n, serr, scratch, s);
            inclusive_scan_u128(nhub, n, serr, scratch, s);
        }
        int64_t hst[4] = {0, 0, 0, 0};
        MC_CUDA(cudaMemcpyAsync(hst, dstat, sizeof(hst), cudaMemcpyDeviceToHost, s));
        u128 tails[2] = {0, 0};
        if (n > 0) {
            MC_CUDA(cudaMemcpyAsync(&tails[0], nch + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(&tails[1], nhub + (n - 1), sizeof(u128), cudaMemcpyDeviceToHost, s));
        }
        MC_CUDA(cudaStreamSynchronize(s));
        MC_REQUIRE(((int *)hst)[0] == 0, "graph is not a canonical symmetric CSR (flags " +
                                             std::to_string(((int *)hst)[0]) +
                                             ": 1 range, 2 loop, 4 order/duplicate, 8 asymmetric)");
        g->max_degree = hst[1];
        g->n_chunks = (int64_t)tails[0];
        g->n_hubs = (int64_t)tails[1];
        MC_REQUIRE(g->n_chunks < (int64_t)0x7fffffff, "too many hub chunks");
        g->chunk_node = g->arena.get<uint32_t>((size_t)g->n_chunks);
        g->chunk_e0 = g->arena.get<int64_t>((size_t)g->n_chunks);
        g->chunk_e1 = g->arena.get<int64_t>((size_t)g->n_chunks);
        g->hub_node = g->arena.get<uint32_t>((size_t)g->n_hubs);
        g->hub_chunk0 = g->arena.get<int64_t>((size_t)g->n_hubs + 1);
        g->node_chunk0 = g->arena.get<int32_t>((size_t)n);
        if (n > 0)
            MC_LAUNCH("hub_chunks", s, hub_chunks<<<grid_for(n, 256), 256, 0, s>>>(
                                           g->row_ptr, n, nch, nhub, g->chunk_node, g->chunk_e0, g->chunk_e1,
                                           g->hub_node, g->hub_chunk0, g->node_chunk0, g->n_hubs, g->n_chunks));
        else
            MC_CUDA(cudaMemsetAsync(g->hub_chunk0, 0, sizeof(int64_t), s));
        g->big_hub = g->arena.get<uint32_t>((size_t)std::max<int64_t>(g->n_hubs, 1));
        unsigned nbig = 0;
        if (g->n_hubs > 0) {
            unsigned *dc = scratch.get<unsigned>(1);
            MC_CUDA(cudaMemsetAsync(dc, 0, sizeof(unsigned), s));
            MC_LAUNCH("big_hubs", s, big_hubs_kernel<<<grid_for(g->n_hubs, 256), 256, 0, s>>>(
                                         g->hub_chunk0, g->n_hubs, dc, g->big_hub));
            MC_CUDA(cudaMemcpyAsync(&nbig, dc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        }
        // the schedule of the neighbour sums: the other nodes by descending degree
        g->n_small = n - g->n_hubs;
        g->sched = g->arena.get<uint4>((size_t)std::max<int64_t>(g->n_small, 1));
        unsigned hh[HUB_CHUNK + 1], cur[HUB_CHUNK + 1];  // live until the synchronisation below
        if (g->n_small > 0) {
            unsigned *dh = scratch.get<unsigned>(2 * (HUB_CHUNK + 1));
            MC_CUDA(cudaMemsetAsync(dh, 0, (HUB_CHUNK + 1) * sizeof(unsigned), s));
            MC_LAUNCH("degree_order", s, degree_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->row_ptr, n, dh));
            MC_CUDA(cudaMemcpyAsync(hh, dh, sizeof(hh), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaStreamSynchronize(s));
            g->n_big_hubs = nbig;
            unsigned run = 0;
            for (int d = HUB_CHUNK; d >= 0; --d) { cur[d] = run; run += hh[d]; }
            MC_REQUIRE((int64_t)run == g->n_small, "degree histogram does not match the hub count");
            MC_CUDA(cudaMemcpyAsync(dh + HUB_CHUNK + 1, cur, sizeof(cur), cudaMemcpyHostToDevice, s));
            MC_LAUNCH("degree_order", s, degree_order_kernel<<<grid_for(n, 256), 256, 0, s>>>(
                                             g->row_ptr, n, dh + HUB_CHUNK + 1, g->sched));
        }
        if (side.done) MC_CUDA(cudaStreamWaitEvent(s, side.done, 0));  // the ids are in place
        MC_CUDA(cudaStreamSynchronize(s));
        g->n_big_hubs = nbig;
    });
    if (st != MC_OK) { delete g; return st; }
    *out = g;
    return MC_OK;
}

extern "C" void mc_free_graph(mc_graph *g) { delete g; }

extern "C" mc_status mc_graph_info(const mc_graph *g, int64_t *n, int64_t *nnz, int64_t *max_degree)
{
    return guarded([&] {
        MC_REQUIRE(g, "graph is NULL");
        if (n) *n = g->n;
        if (nnz) *nnz = g->nnz;
        if (max_degree) *max_degree = g->max_degree;
    });
}

extern "C" mc_status mc_color(const mc_graph *g, int k, uint64_t seed, uint8_t *colors, void *stream)
{
    return guarded([&] {
        MC_REQUIRE(g && colors, "graph or colors is NULL");
        MC_REQUIRE(k >= 1 && k <= 255, "k out of range");
        if (g->n == 0) return;
        cudaStream_t s = (cudaStream_t)stream;
        MC_LAUNCH("color", s, color_kernel<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, k, seed, colors));
    });
}

extern "C" mc_status mc_color_biased(const mc_graph *g, int k, uint64_t seed, uint32_t lambda_q32, uint8_t *colors,
                                     void *stream)
{
    if (lambda_q32 == 0) return mc_color(g, k, seed, colors, stream);
    return guarded([&] {
        MC_REQUIRE(g && colors, "graph or colors is NULL");
        MC_REQUIRE(k >= 2 && k <= 255, "k out of range");
        MC_REQUIRE((uint64_t)(k - 1) * lambda_q32 <= 4294967296ull, "(k-1) lambda must be at most 1");
        if (g->n == 0) return;
        cudaStream_t s = (cudaStream_t)stream;
        MC_LAUNCH("color", s, color_biased_kernel<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, k, seed, lambda_q32,
                                                                                      colors));
    });
}
