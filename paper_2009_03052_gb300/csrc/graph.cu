// graph.cu -- error plumbing, device memory, graph loading and validation,
// colouring (Section 2.1).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace mc {

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

void Arena::release_all()
{
    for (auto &b : blocks) alloc.release(b.first, b.second, stream);
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

// ---------------------------------------------------------------------------
// tracing
// ---------------------------------------------------------------------------
namespace {
struct ProfState {
    std::mutex mu;
    bool on = false;
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int64_t> launches;
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
    });
}

extern "C" mc_status mc_profile_read(char *names, size_t names_bytes, double *ms, int64_t *launches, int max,
                                     int *count)
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
        const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        g->row_ptr = g->arena.get<int64_t>((size_t)n + 1);
        g->col = g->arena.get<uint32_t>((size_t)(nnz > 0 ? nnz : 1));
        MC_CUDA(cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int64_t) * (n + 1), kind, s));
        if (nnz) MC_CUDA(cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * nnz, kind, s));
        // host copy of the offsets, for degree statistics and hub chunks
        std::vector<int64_t> rp((size_t)n + 1);
        MC_CUDA(cudaMemcpyAsync(rp.data(), g->row_ptr, sizeof(int64_t) * (n + 1),
                                cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        MC_REQUIRE(rp[0] == 0 && rp[n] == nnz, "row_ptr[0] must be 0 and row_ptr[n] must be nnz");
        // offsets are checked here, before any kernel indexes with them
        for (int64_t v = 0; v < n; ++v)
            MC_REQUIRE(rp[v] <= rp[v + 1], "row_ptr must be non-decreasing");
        if (!(flags & MC_GRAPH_TRUSTED) && n > 0) {
            int *dflags = g->arena.get<int>(1);
            MC_CUDA(cudaMemsetAsync(dflags, 0, sizeof(int), s));
            if (nnz)
                MC_LAUNCH("validate_edges", s,
                          validate_edges<<<grid_for(nnz, 256), 256, 0, s>>>(g->row_ptr, g->col, n, nnz, dflags));
            int hf = 0;
            MC_CUDA(cudaMemcpyAsync(&hf, dflags, sizeof(int), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaStreamSynchronize(s));
            MC_REQUIRE(hf == 0, "graph is not a canonical symmetric CSR (flags " + std::to_string(hf) +
                                    ": 1 range, 2 loop, 4 order/duplicate, 8 asymmetric)");
        }
        // degree statistics and hub chunks
        std::vector<uint32_t> cn, hn;
        std::vector<int64_t> c0, c1, h0;
        for (int64_t v = 0; v < n; ++v) {
            const int64_t d = rp[v + 1] - rp[v];
            g->max_degree = std::max(g->max_degree, d);
            if (d > HUB_CHUNK) {
                hn.push_back((uint32_t)v);
                h0.push_back((int64_t)cn.size());
                for (int64_t e = rp[v]; e < rp[v + 1]; e += HUB_CHUNK) {
                    cn.push_back((uint32_t)v);
                    c0.push_back(e);
                    c1.push_back(std::min(e + HUB_CHUNK, rp[v + 1]));
                }
            }
        }
        h0.push_back((int64_t)cn.size());
        MC_REQUIRE(cn.size() < (size_t)0x7fffffff, "too many hub chunks");
        std::vector<int32_t> nc0((size_t)n, -1);
        for (size_t i = 0; i < hn.size(); ++i) nc0[hn[i]] = (int32_t)h0[i];
        g->node_chunk0 = g->arena.get<int32_t>((size_t)n);
        if (n) MC_CUDA(cudaMemcpyAsync(g->node_chunk0, nc0.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        g->n_hubs = (int64_t)hn.size();
        g->n_chunks = (int64_t)cn.size();
        g->chunk_node = g->arena.get<uint32_t>(cn.size());
        g->chunk_e0 = g->arena.get<int64_t>(c0.size());
        g->chunk_e1 = g->arena.get<int64_t>(c1.size());
        g->hub_node = g->arena.get<uint32_t>(hn.size());
        g->hub_chunk0 = g->arena.get<int64_t>(h0.size());
        if (!cn.empty()) {
            MC_CUDA(cudaMemcpyAsync(g->chunk_node, cn.data(), cn.size() * 4, cudaMemcpyHostToDevice, s));
            MC_CUDA(cudaMemcpyAsync(g->chunk_e0, c0.data(), c0.size() * 8, cudaMemcpyHostToDevice, s));
            MC_CUDA(cudaMemcpyAsync(g->chunk_e1, c1.data(), c1.size() * 8, cudaMemcpyHostToDevice, s));
            MC_CUDA(cudaMemcpyAsync(g->hub_node, hn.data(), hn.size() * 4, cudaMemcpyHostToDevice, s));
        }
        MC_CUDA(cudaMemcpyAsync(g->hub_chunk0, h0.data(), h0.size() * 8, cudaMemcpyHostToDevice, s));
        MC_CUDA(cudaStreamSynchronize(s));
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
