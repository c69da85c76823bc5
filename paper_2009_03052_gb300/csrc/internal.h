// internal.h -- handle layouts, error plumbing and device memory helpers of
// libmotif (host side).
#pragma once

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/motif.h"
#include "catalog.h"
#include "common.cuh"

namespace mc {

// An error carrying an mc_status; caught at the ABI boundary.
struct Error : std::runtime_error {
    mc_status status;
    Error(mc_status s, const std::string &what) : std::runtime_error(what), status(s) {}
};

void set_last_error(const std::string &msg);

#define MC_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            throw ::mc::Error(MC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define MC_REQUIRE(cond, msg)                                        \
    do {                                                             \
        if (!(cond)) throw ::mc::Error(MC_E_INVALID, msg);           \
    } while (0)

// Device memory through the caller's allocator (or cudaMalloc).
struct Allocator {
    mc_allocator a{};
    bool custom = false;
    void *alloc(size_t bytes, cudaStream_t s) const;
    void release(void *p, size_t bytes, cudaStream_t s) const;
};

// A set of device buffers released together.  A scratch arena (buffers of
// one call, used on its stream only) takes stream-ordered memory
// (cudaMallocAsync) when no allocator is given, so concurrent calls on
// different streams never synchronise the device to allocate.
struct Arena {
    Allocator alloc;
    cudaStream_t stream = nullptr;
    bool scratch = false;
    std::vector<std::pair<void *, size_t>> blocks;
    Arena() = default;
    explicit Arena(bool is_scratch) : scratch(is_scratch) {}
    template <typename T> T *get(size_t count)
    {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 256;
        void *p = nullptr;
        if (scratch && !alloc.custom) {
            if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
        } else {
            p = alloc.alloc(bytes, stream);
        }
        if (!p) throw Error(MC_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        blocks.emplace_back(p, bytes);
        return static_cast<T *>(p);
    }
    void release_all();
    void release(void *p);  // one block, by its pointer
    ~Arena() { release_all(); }
};

// Run f, turning exceptions into an mc_status and mc_last_error().
template <typename F> mc_status guarded(F &&f)
{
    try {
        f();
        return MC_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return MC_E_NOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return MC_E_INTERNAL;
    }
}

int grid_for(int64_t work, int block);
int sm_count();

// Kernel tracing: count every launch; when profiling is on, bracket it by
// CUDA events on its stream, keyed by a kernel name.
struct ProfSpan {
    cudaEvent_t a = nullptr, b = nullptr;
    int id = -1;
};
bool prof_enabled();
bool prof_counting();
void prof_add_bytes(const char *name, int64_t bytes);
ProfSpan prof_begin(const char *name, cudaStream_t s);
void prof_end(ProfSpan &span, cudaStream_t s);

#define MC_LAUNCH(name, stream, ...)                                  \
    do {                                                              \
        ::mc::ProfSpan sp_ = ::mc::prof_begin(name, stream);          \
        __VA_ARGS__;                                                  \
        cudaError_t le_ = cudaGetLastError();                         \
        ::mc::prof_end(sp_, stream);                                  \
        if (le_ != cudaSuccess)                                       \
            throw ::mc::Error(MC_E_CUDA, std::string(name) + ": " + cudaGetErrorString(le_)); \
    } while (0)

// Make sure level h's root index (node prefix of the level totals, R and
// the root-search buckets) exists; builds and publishes it on first use.
void ensure_level_index(const mc_tables *t, int h, cudaStream_t s);
// After mc_rebuild_tables: read the new level-k total and bucket width and
// the error flags back (synchronises s); throws if the rebuild failed.
// force: re-read even without a rebuild through the API (a replayed graph).
void refresh_tables(const mc_tables *t, cudaStream_t s, bool force = false);
// Copies of unrooted shape j from its rooted total R at level h: R / h, R at
// a zero-rooted level k, R / a_j at a round-skipped level k (0 for the star).
u128 unrooted_from_rooted(const mc_tables *t, int h, int j, u128 R);
// Replace every dense c and S level of t by its packed form (synchronises s).
void pack_tables(mc_tables *t, cudaStream_t s);
// Per-node totals over the allowed shapes of packed level h of c.
void launch_packed_row_totals(const mc_tables *t, int h, uint64_t allow0, uint64_t allow1, u128 *tot, int *err,
                              cudaStream_t s);
// Expand packed level h (which = 0: c, 1: S) into a dense n x W table.
void launch_unpack(const mc_tables *t, int h, int which, void *dst, cudaStream_t s);

// Warp tasks of the neighbour-sum kernel: a node with more than HUB_CHUNK
// neighbours is split into chunks of HUB_CHUNK consecutive neighbours whose
// sums are added afterwards (and kept as their prefix for the sampler).
constexpr int HUB_CHUNK = 64;
// Hubs of at most HUB_SERIAL chunks have their chunk sums added up by one
// thread per S entry; larger ones (listed in big_hub) by a warp per entry.
constexpr int HUB_SERIAL = 32;

}  // namespace mc

struct mc_tables;
struct mc_graph {
    int64_t n = 0, nnz = 0, max_degree = 0;
    int64_t *row_ptr = nullptr;  // device int64[n+1]
    uint32_t *col = nullptr;     // device uint32[nnz]
    // hub chunks (device): node, first edge, end edge; per hub, its first chunk
    int64_t n_chunks = 0, n_hubs = 0;
    uint32_t *chunk_node = nullptr;
    int64_t *chunk_e0 = nullptr, *chunk_e1 = nullptr;
    uint32_t *hub_node = nullptr;
    int64_t *hub_chunk0 = nullptr;  // n_hubs + 1 entries
    int32_t *node_chunk0 = nullptr; // per node: its first chunk if it is a hub, else -1
    // the nodes of degree <= HUB_CHUNK in descending order of degree (the
    // schedule of the neighbour-sum kernel), n_small of them, one record each:
    // (node, first edge low word, first edge high word, degree)
    uint4 *sched = nullptr;
    int64_t n_small = 0;
    uint32_t *big_hub = nullptr;  // hubs (indices into hub_node) of more than HUB_SERIAL chunks
    int64_t n_big_hubs = 0;
    mc::Arena arena;
    // uncoloured h-star index, built on first use: inclusive prefix over v of
    // C(d_v, h-1) and its total
    std::mutex star_mu;
    mc::u128 *star_prefix[mc::MAXK + 1] = {nullptr};
    mc::u128 star_total[mc::MAXK + 1] = {0};
    uint32_t *star_bucket[mc::MAXK + 1] = {nullptr};  // bucket index of the prefix (as for roots)
    mc::u128 star_D[mc::MAXK + 1] = {0};
};

struct mc_tables {
    const mc_graph *g = nullptr;
    mc_graph *owned_graph = nullptr;  // the union graph of a batch build, freed with the tables
    int k = 0, bits = 64;
    bool zero_root = false;  // level k stored at colour-0 nodes only
    // copies per stored level-h entry sum: h, or 1 for a zero-rooted level k
    int copies_div(int h) const { return (zero_root && h == k) ? 1 : h; }
    bool skip_round = false;  // level k-1 skipped, level k by balanced decompositions
    int copies_k[32] = {0};   // with skip_round: a_j per unrooted k-shape (0: the star)
    bool level_missing(int h) const { return h < 1 || h > k || (skip_round && h == k - 1); }
    mc::Geometry geo;
    uint8_t *colors = nullptr;                 // device uint8[n]
    uint8_t *ecol = nullptr;                   // device uint8[nnz]: colour of col[e]
    uint32_t *scol = nullptr;                  // device uint32[nnz]: each node's neighbours grouped
                                               // by colour, ascending ids inside a colour
    int32_t *coff = nullptr;                   // device int32[n*(k+1)]: start of colour a's block in
                                               // v's row of scol, relative to row_ptr[v]
    void *c[mc::MAXK + 1] = {nullptr};         // level h >= 2: n x Wc[h] counts
    void *S[mc::MAXK + 1] = {nullptr};         // level h <= k-1: n x Ws[h] counts
    void *Sp[mc::MAXK + 1] = {nullptr};        // level h <= k-1: per hub and S entry, the inclusive
                                               // prefix of its chunk sums, n_chunks x Ws[h]
    mc::u128 *prefix[mc::MAXK + 1] = {nullptr};  // inclusive node prefix of level totals
    mc::u128 R[mc::MAXK + 1] = {0};            // rooted totals
    // root index of a level (node prefix, R, buckets): level k at build,
    // other levels on first use (guarded by idx_mu)
    std::mutex idx_mu;
    uint32_t *bucket[mc::MAXK + 1] = {nullptr}; // root-search buckets over [0, R) (see sample.cu)
    mc::u128 bucketD[mc::MAXK + 1] = {0};
    int64_t nbucket = 0;
    // merge and gather programs (device)
    int32_t *m_info[mc::MAXK + 1] = {nullptr};
    int32_t *m_off[mc::MAXK + 1] = {nullptr};
    uint32_t *m_terms[mc::MAXK + 1] = {nullptr};
    int16_t *g_map[mc::MAXK + 1] = {nullptr};
    // kept for in-place rebuilds (mc_rebuild_tables): error flags, hub colour
    // counts, scan tile sums and the bucket width of level k, all on the device
    int *dev_err = nullptr;
    uint32_t *ccnt = nullptr;
    mc::u128 *scan_tmp = nullptr;
    mc::u128 *dev_D = nullptr;
    // packed levels (MC_BUILD_SUCCINCT / MC_BUILD_VARLEN): the dense c[h] and
    // S[h] are freed once packed; pc / ps hold the levels instead
    bool packed = false, varlen = false;
    mc::PackedView pc[mc::MAXK + 1], ps[mc::MAXK + 1];
    int64_t dense_bytes = 0, stored_bytes = 0;  // of the c and S levels
    bool stale = false;                         // rebuilt since R[k], bucketD[k] were read back
    bool level_stale[mc::MAXK + 1] = {false};   // root index of level h from an older colouring
    std::string broken;                         // set when a rebuild failed its checks
    mc::Arena arena;
};
