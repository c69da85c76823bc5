/*
 * motif.h -- C ABI of the GB300 colour-coding motif library (libmotif).
 *
 * Colour coding for k-node graphlet counting after Bressan, Leucci and
 * Panconesi, "Faster motif counting via succinct color coding and adaptive
 * sampling": colour the graph (Section 2.1), build the exact colourful
 * treelet count tables c(T_C, v) by the dynamic program of Eq. (1), sample
 * colourful treelets uniformly (Section 2.2) or adaptively (Algorithm AGS,
 * Section 4.1), classify the induced graphlets (Section 4.4.3) and estimate
 * graphlet counts.
 *
 * Conventions for every entry point:
 *  - Pointers named "device" must point to device memory of the current CUDA
 *    device; "host" pointers to host memory.  The caller owns every pointer it
 *    passes; the library owns the handles it returns and frees them in
 *    mc_free_*.  Device work is queued on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  Entry points that return host results
 *    synchronise `stream` before returning.
 *  - Every entry point returns an mc_status.  On error no handle is returned,
 *    nothing the caller owns is freed, and mc_last_error() (per host thread)
 *    says why.  No C++ exception crosses the ABI.
 *  - Counts are exact unsigned integers of 64 or 128 bits.  An intermediate
 *    value that does not fit the count width (a table entry, a neighbour sum,
 *    a merge numerator or a level total) makes the call fail with
 *    MC_E_OVERFLOW; nothing wraps.
 *  - Graphs are simple and undirected (Section 1.3): n < 2^32 nodes, CSR with
 *    symmetric, sorted, duplicate-free, loop-free adjacency lists.
 *  - 2 <= k <= 8 colours; treelets and graphlets have h <= k nodes.
 */
#ifndef MOTIF_H
#define MOTIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MC_OK = 0,
    MC_E_INVALID = 1,      /* bad argument or malformed graph */
    MC_E_NOMEM = 2,        /* the allocator returned NULL */
    MC_E_OVERFLOW = 3,     /* a count does not fit the chosen width */
    MC_E_CUDA = 4,         /* a CUDA runtime call failed */
    MC_E_TIMEOUT = 5,      /* reserved: a bounded device wait gave up */
    MC_E_UNSUPPORTED = 6,  /* valid but not supported (e.g. k > 8) */
    MC_E_INTERNAL = 7      /* an internal consistency check failed */
} mc_status;

/* Device memory provider.  alloc returns device memory of at least `bytes`
 * bytes, aligned to 256 bytes, usable on `stream` (NULL on failure); free
 * releases it.  `ctx` is passed back unchanged and must outlive every handle
 * created with this allocator.  A NULL allocator means cudaMalloc/cudaFree. */
typedef struct mc_allocator {
    void *(*alloc)(size_t bytes, void *ctx, void *stream);
    void (*free)(void *ptr, size_t bytes, void *ctx, void *stream);
    void *ctx;
} mc_allocator;

typedef struct mc_graph mc_graph;
typedef struct mc_tables mc_tables;

/* ------------------------------------------------------------------------ */
/* Graph                                                                     */
/* ------------------------------------------------------------------------ */
#define MC_GRAPH_DEVICE_PTRS 0x1u  /* row_ptr and col are device pointers */
#define MC_GRAPH_TRUSTED     0x2u  /* skip the canonical-CSR validation */

/* Copy a CSR graph to the device.  row_ptr: int64[n+1] with row_ptr[0] = 0
 * and row_ptr[n] = nnz; col: uint32[nnz], node u's neighbours are
 * col[row_ptr[u] .. row_ptr[u+1]) in strictly ascending order.  Unless
 * MC_GRAPH_TRUSTED is set the copy is checked on the device (bounds, order,
 * no loops, symmetry) and a malformed graph gives MC_E_INVALID.  The input
 * buffers are not retained. */
mc_status mc_load_graph(int64_t n, int64_t nnz, const int64_t *row_ptr, const uint32_t *col,
                        uint32_t flags, const mc_allocator *alloc, void *stream, mc_graph **out);
void mc_free_graph(mc_graph *g);
/* n, nnz (= 2m) and the largest degree. */
mc_status mc_graph_info(const mc_graph *g, int64_t *n, int64_t *nnz, int64_t *max_degree);

/* ------------------------------------------------------------------------ */
/* Colouring (Section 2.1: every node draws a colour uniformly from [k])     */
/* ------------------------------------------------------------------------ */
/* colors: device uint8[n], written.  c_v = floor(k * x0 / 2^32) with x0 the
 * first word of Philox4x32-10 (Salmon et al., SC 2011) at key = seed
 * (low word first) and counter = (v, 0, 0, 0xC010). */
mc_status mc_color(const mc_graph *g, int k, uint64_t seed, uint8_t *colors, void *stream);
/* Biased colouring (Section 3.5): colours 1..k-1 each with probability
 * lambda = lambda_q32 / 2^32, colour 0 with 1 - (k-1) lambda ((k-1) lambda
 * <= 1, else MC_E_INVALID).  Same counter and key as mc_color; x0 the first
 * output word: c_v = 1 + floor(x0 / lambda_q32) when x0 < (k-1) lambda_q32,
 * else 0.  lambda_q32 = 0 is mc_color.  Estimates from tables built with
 * such colours must be given the same lambda_q32 (colour_bias_q32 of
 * mc_estimate_params). */
mc_status mc_color_biased(const mc_graph *g, int k, uint64_t seed, uint32_t lambda_q32, uint8_t *colors,
                          void *stream);

/* ------------------------------------------------------------------------ */
/* Count tables (Section 2.1, Eq. 1; Section 3.2.1)                          */
/* ------------------------------------------------------------------------ */
/* Build c(T_C, v) for every rooted treelet shape T on h = 1..k nodes, every
 * colour set C with |C| = h and every node v, by the dynamic program of
 * Eq. (1) split in two steps per level: the neighbour sums
 * S(T'', C'', v) = sum_{u ~ v} c(T''_{C''}, u) and the disjoint-colour merge
 * c(T_C, v) = (1/beta_T) sum_{C' + C'' = C} c(T'_{C'}, v) S(T'', C'', v).
 * colors: device uint8[n] with values < k (read during the call only).
 * count_bits: 64 or 128.  flags: 0 or MC_BUILD_ZERO_ROOT or MC_BUILD_SKIP_ROUND, each
 * optionally with MC_BUILD_SUCCINCT or MC_BUILD_VARLEN.  The tables stay on the device
 * until mc_free_tables; they are immutable, so concurrent readers are safe.
 * The graph must outlive the tables. */
/* Zero-rooting (Section 3.4.1): keep the level-k counts only at nodes of
 * colour 0 (zero elsewhere).  Every colourful k-treelet has exactly one
 * colour-0 node, so level k then holds each copy once: its total is t itself
 * (not h t), and sampling at h = k draws the root among colour-0 nodes, still
 * uniformly over the copies. */
#define MC_BUILD_ZERO_ROOT 0x1u
/* Round skipping (Section 3.3.2), k >= 4, not with zero-rooting: level k is
 * built from a balanced decomposition -- T'' the subtree of the first root
 * child (in s_T order) with 2..k-2 nodes, T' the rest, beta_T the root
 * children equal to T'' -- so level k-1 is never built (its tables,
 * totals, samples and reads are MC_E_INVALID).  Rooted k-shapes without such
 * a child (the star rooted anywhere, every leaf rooting) are not counted:
 * their level-k entries are 0.  A copy of tree j then appears once per node
 * at which its rooting is counted (a_j of them; 0 for the k-star), so
 * mc_total(k, j) returns R_j and t_j = R_j / a_j (0 for the star), and the
 * all-shapes total returns R and sum_j t_j.  k-stars are sampled uncoloured
 * with mc_sample_stars and estimated from those samples (star_samples in
 * mc_estimate_params). */
#define MC_BUILD_SKIP_ROUND 0x2u
/* Succinct tables (Section 3.2.1): once built, every level of c and S is
 * kept as its non-zero entries only -- per node row, the entries' keys (their
 * index in the dense row of mc_table_layout) in ascending order and their
 * counts at the table's width -- and the dense levels are freed.  Sampling
 * finds an entry by binary search of its row's keys; results are the same as
 * from dense tables.  mc_read_table still returns dense rows;
 * mc_table_nonzeros is the packed size; mc_table_bytes reports the
 * footprint.  Such tables cannot be rebuilt in place (MC_E_UNSUPPORTED). */
#define MC_BUILD_SUCCINCT 0x4u
/* Variable-length counts (Section 3.3.3), implies MC_BUILD_SUCCINCT: each
 * packed row stores its counts in the fewest of 1, 2, 4, 8 or 16 bytes that
 * hold the row's largest count (the paper gives each count its own byte
 * length; a per-row width keeps every load aligned). */
#define MC_BUILD_VARLEN 0x8u

mc_status mc_build_tables(const mc_graph *g, const uint8_t *colors, int k, int count_bits,
                          uint32_t flags, const mc_allocator *alloc, void *stream,
                          mc_tables **out);
/* Device bytes of the c and S levels: as dense rows (n x row entries x count
 * bytes per level) and as stored (the same for dense tables; keys, counts and
 * row offsets for succinct ones).  Host int64 outputs, either may be NULL. */
mc_status mc_table_bytes(const mc_tables *t, int64_t *dense_bytes, int64_t *stored_bytes);
void mc_free_tables(mc_tables *t);

/* Totals (the occ() queries of Section 3): rooted = sum over v and over the
 * rooted shapes of size h (all of them when unrooted_shape < 0, else the
 * rootings of that unrooted shape) of the stored c(T_C, v); unrooted = the
 * number of colourful h-treelet copies t (or t_j): rooted / h, or rooted
 * itself for a zero-rooted level k.  Host uint64[2] each, low word first.
 * Synchronises `stream`. */
mc_status mc_total(const mc_tables *t, int h, int32_t unrooted_shape, uint64_t rooted[2],
                   uint64_t unrooted_count[2], void *stream);
/* The same over the treelets rooted at nodes [node_lo, node_hi) (node_hi <= 0:
 * to the last node), e.g. one instance of a batch. */
mc_status mc_total_range(const mc_tables *t, int h, int32_t unrooted_shape, int64_t node_lo, int64_t node_hi,
                         uint64_t rooted[2], uint64_t unrooted_count[2], void *stream);

/* Batches (many colourings of one graph, many graphs): build the tables of
 * `count` independent (graph, colouring) instances in one pass.  The
 * instances are laid side by side as one disjoint union, so every kernel of
 * the build is launched once for the whole batch; instance i owns the union's
 * nodes [node_offsets[i], node_offsets[i+1]) (host int64[count+1], written),
 * its node v being union node node_offsets[i] + v with the same neighbour
 * order.  Treelets never cross instances, so every count, total and sample
 * of instance i (queried with its node range) equals that of its own
 * mc_build_tables, with node ids shifted by node_offsets[i].  The graphs and
 * colour buffers are read during the call only. */
mc_status mc_build_tables_batch(int count, const mc_graph *const *graphs, const uint8_t *const *colors, int k,
                                int count_bits, uint32_t flags, const mc_allocator *alloc, void *stream,
                                mc_tables **out, int64_t *node_offsets);

/* Rebuild t in place for a new colouring (device or host uint8[n], values
 * < k): the same graph, k, count width and flags; every buffer of the first
 * build is reused.  The call allocates nothing, only enqueues kernels,
 * memsets and one copy of the colours on `stream`, and never synchronises,
 * so it can be captured into a CUDA graph and replayed (write the next
 * colouring into the same buffer before each replay; colors == the tables'
 * own colour buffer skips the copy).  Checks (a colour >= k, overflow) are
 * recorded on the device and reported by the next call that reads the
 * tables (mc_total, mc_sample, mc_estimate_counts, mc_read_table) or by
 * mc_tables_status, which also reads the new level-k total back
 * (synchronising `stream`); issue them on the rebuild's stream or after
 * synchronising it.  A replay of a captured rebuild runs no host code: call
 * mc_tables_status after each replay before any other call on t.  mc_estimate_uniform_noalloc after a rebuild needs
 * mc_tables_status first.  Root indices of levels below k made by earlier
 * calls are rebuilt on first use.  No other call may use t while a rebuild
 * is in flight.  The paper has no counterpart: it builds once per
 * colouring. */
mc_status mc_rebuild_tables(mc_tables *t, const uint8_t *colors, void *stream);
mc_status mc_tables_status(const mc_tables *t, void *stream);

/* Autotuning of the build's kernel schedules (no counterpart in the paper:
 * the choice of GPU schedule).  The neighbour-sum and merge kernels of each
 * level have a few schedules (lanes per node, rows in flight, registers per
 * thread) that compute identical tables.  mc_build_tables times
 * every candidate once for each new (kernel, k, count width, level, degree
 * bucket) key and keeps the fastest; the degree bucket is floor(log2 n),
 * floor(2 log2(nnz / n)) and floor(log2(max degree + 1)).  mc_rebuild_tables
 * never tunes (it may be captured): it uses the choices made so far.
 *   mode 0: never tune (choices loaded or made earlier, else the first
 *           schedule); 1 (default): tune keys not seen yet; 2: tune every key
 *           once more in this process.
 *   cache_file (may be NULL: unchanged; "": stop appending): load its
 *   choices now and append every new one to it; the MC_AUTOTUNE_CACHE
 *   environment variable does the same at the first build.  One line per key: kind k bits h logn logdeg loghub choice.
 * mc_autotune_choice: the schedule chosen so far for kernel kind (0 the
 * neighbour sums, schedules 0..6; 1 the merge, schedules 0..5) at level h
 * of tables with k colours and count_bits counts on graphs of n nodes, nnz
 * adjacency entries and largest degree max_degree (mc_graph_info), or -1.
 * mc_autotune_set: fix that choice (MC_E_INVALID for an unknown kind or
 * schedule); builds use it and do not tune it again (in mode 1). */
mc_status mc_autotune(int mode, const char *cache_file);
int mc_autotune_choice(int kind, int k, int count_bits, int h, int64_t n, int64_t nnz, int64_t max_degree);
mc_status mc_autotune_set(int kind, int k, int count_bits, int h, int64_t n, int64_t nnz, int64_t max_degree,
                          int choice);

/* Layout of the level-h table (which = 0: counts c, h = 1..k; which = 1:
 * neighbour sums S, h = 1..k-1).  Row v holds row_entries entries of
 * entry_bytes (8 or 16, little-endian, low word first).  Rows are
 * set-major: entry (rho, s) sits at rho * r_h + s, s the rooted shape id,
 * r_h = mc_num_shapes(h), and rho the colex rank (among C(k-1, h-1) sets for
 * c, C(k-1, h) for S) of the colour set without c_v after deleting colour
 * c_v from the palette (colours above c_v move down by one).  Only sets that
 * contain c_v (for c) or avoid it (for S) are stored. */
mc_status mc_table_layout(const mc_tables *t, int h, int which, int64_t *row_entries,
                          int *entry_bytes);
/* Non-zero entries of a level (which = 0: c, which = 1: S), counted on the
 * device: the entries a zero-suppressed (succinct) table would keep
 * (Section 3.2.1).  Synchronises `stream`. */
mc_status mc_table_nonzeros(const mc_tables *t, int h, int which, int64_t *count, void *stream);

/* Copy a whole level (n * row_entries * entry_bytes bytes) into dst (host or
 * device as dst_on_device says).  Level 1 of c is all ones and is produced on
 * the fly.  Synchronises `stream`. */
mc_status mc_read_table(const mc_tables *t, int h, int which, void *dst, size_t dst_bytes,
                        int dst_on_device, void *stream);

/* ------------------------------------------------------------------------ */
/* Sampling (Section 2.2; sample(T) of Section 4.1)                          */
/* ------------------------------------------------------------------------ */
/* Draw `count` colourful h-treelets (2 <= h <= k) uniformly among all
 * copies (unrooted_shape < 0) or among the copies of one unrooted shape,
 * with sample indices first_index, first_index + 1, ...  Sample i is a pure
 * function of (tables, seed, i), so batches can be split or reordered freely.
 * Outputs (device; any may be NULL): nodes uint32[count*h] (each sample's
 * nodes ascending), roots uint32[count], shapes int32[count] (rooted shape
 * id), classes int32[count] (id of the induced h-node graphlet: rank of its
 * canonical adjacency word among those of all connected h-node graphs).
 * MC_E_INVALID when no such treelet exists. */
mc_status mc_sample(const mc_tables *t, int h, int32_t unrooted_shape, uint64_t seed,
                    uint64_t first_index, int64_t count, uint32_t *nodes, uint32_t *roots,
                    int32_t *shapes, int32_t *classes, void *stream);
/* The same restricted to the treelets rooted at nodes [node_lo, node_hi) --
 * for a batch instance, exactly its own samples (node ids in the union's
 * numbering). */
mc_status mc_sample_range(const mc_tables *t, int h, int32_t unrooted_shape, int64_t node_lo, int64_t node_hi,
                          uint64_t seed, uint64_t first_index, int64_t count, uint32_t *nodes,
                          uint32_t *roots, int32_t *shapes, int32_t *classes, void *stream);

/* Uncoloured h-stars (Section 3.3.2), 2 <= h <= 8, drawn uniformly among
 * all h-stars of the graph: sample i takes the centre v with probability
 * C(d_v, h-1) / S, S = sum_v C(d_v, h-1), then h-1 distinct neighbours of v
 * uniformly.  Random numbers: counter (i_lo, i_hi, 16, attempt) gives
 * X = uniform(S) and v is the first node whose inclusive prefix of
 * C(d_u, h-1) exceeds X; counter (i_lo, i_hi, 17 + s, attempt), s = 0..h-2,
 * gives x = uniform(d_v - s) and the x-th neighbour position, ascending,
 * among those not yet taken.  Outputs (device; any may be NULL): nodes
 * uint32[count*h] ascending, centres uint32[count], classes int32[count]
 * (graphlet class of the induced subgraph, as for mc_sample).  The star
 * index (16 bytes per node and h) is built on first use and kept with the
 * graph.  MC_E_INVALID when the graph has no h-star, MC_E_OVERFLOW when S
 * does not fit in 128 bits. */
mc_status mc_star_total(const mc_graph *g, int h, uint64_t total[2], void *stream);
mc_status mc_sample_stars(const mc_graph *g, int h, uint64_t seed, uint64_t first_index, int64_t count,
                          uint32_t *nodes, uint32_t *centres, int32_t *classes, void *stream);

/* ------------------------------------------------------------------------ */
/* Estimation (Section 2.2 uniform; Algorithm AGS, Section 4.1)              */
/* ------------------------------------------------------------------------ */
#define MC_EST_UNIFORM 0
#define MC_EST_AGS 1

typedef struct {
    int mode;              /* MC_EST_UNIFORM or MC_EST_AGS */
    int h;                 /* graphlet size, 2 <= h <= k */
    uint64_t seed;
    uint64_t first_index;  /* uniform: sample s has index first_index + s; AGS: every
                              treelet shape j has its own stream, the n-th sample drawn
                              with T_j has index first_index + j * 2^40 + n */
    int64_t samples;       /* uniform: samples drawn; AGS: the most it may draw (<= 2^40,
                              else MC_E_INVALID) */
    int64_t cbar;          /* AGS covering threshold; <= 0: ceil(4/eps^2 ln(2s/delta)) */
    double eps, delta;     /* AGS accuracy, used when cbar <= 0 */
    int64_t batch;         /* AGS: samples drawn ahead for the current treelet per launch
                              (and min(batch, 4096) for each other treelet whose drawn-ahead
                              samples are used up); <= 0: automatic.  The result does not
                              depend on it */
    int64_t node_lo, node_hi;  /* root nodes [node_lo, node_hi); node_hi <= 0: all nodes */
    uint32_t colour_bias_q32;  /* lambda_q32 of the biased colouring the tables were built with
                                  (0: uniform); the estimate divides by the probability
                                  p = h! (C(k-1,h) lambda^h + C(k-1,h-1) lambda^(h-1) (1-(k-1) lambda))
                                  that an h-node set is colourful, evaluated in that order in
                                  double */
    int64_t star_samples;  /* round-skipped tables at h = k: uncoloured h-stars drawn (with the
                              same sample indices) to estimate the graphlets that only stars
                              span; their estimate is (S * hits*_i) / (sigma*_i * star_samples),
                              S the h-stars of G, sigma*_i the spanning stars of H_i, and their
                              hits are the star hits (0 star samples: estimate 0) */
} mc_estimate_params;

typedef struct {
    int64_t samples;    /* samples that entered the estimate */
    int64_t switches;   /* AGS: treelet switches */
    int64_t covered;    /* AGS: graphlets covered */
    int64_t batches;    /* device batches launched */
    int64_t discarded;  /* AGS: samples drawn ahead and not used */
} mc_estimate_stats;

/* est: host double[N_h], the estimated number of induced copies of each
 * h-node graphlet in G; hits: host uint64[N_h], samples per graphlet;
 * stats: host, may be NULL.  N_h = mc_num_classes(h).  Synchronises.  AGS
 * page-locks a host buffer of about 4 (B + 4096 U) bytes (B = batch, or 2^22
 * when automatic; U = mc_num_unrooted(h)) that the calling thread keeps for
 * its later calls and frees when it exits. */
mc_status mc_estimate_counts(const mc_tables *t, const mc_estimate_params *params, double *est,
                             uint64_t *hits, mc_estimate_stats *stats, void *stream);

/* Uniform estimation that allocates no device memory, for callers that
 * cannot allocate: serving loops that hand every byte of device memory to
 * their own pool up front (a cudaMalloc would fail or take memory the pool
 * counts on), and latency-critical loops that must not hit cudaMalloc's
 * implicit device synchronisation.  The paper has no counterpart: it
 * computes the same result as mc_estimate_counts in MC_EST_UNIFORM mode
 * (same samples, same hits, same estimates).
 *  - Its device scratch (histogram, sigma and estimate arrays, error flags)
 *    is one static array of the library, sized for at most 12288 graphlet
 *    classes (about 290 KB), which every GPU that loads the library holds
 *    until the process exits.  Classes beyond that limit give
 *    MC_E_UNSUPPORTED (the largest supported size, h = 8, has 11117).
 *  - The first call on a device looks up that array's device address (no
 *    allocation); make that first call before any stream capture.
 *  - The graphlet catalogue of size h must already exist on the device
 *    (mc_sigma(h), mc_num_classes(h) with mc_sigma, or mc_estimate_counts
 *    create it); otherwise MC_E_INVALID, since creating it allocates.  For
 *    h < k the same holds for the level's root index (mc_total(t, h, -1, ...)
 *    or any sampling at that h creates it), and after mc_rebuild_tables an
 *    index of such a level made before the rebuild is refused with
 *    MC_E_INVALID until mc_total(t, h, ...) remakes it.
 *  - All calls share the one scratch array, cleared at the start of each
 *    call: calls whose work overlaps on the GPU (other streams, other host
 *    threads) race and must be serialised by the caller.
 * est, hits: host arrays of mc_num_classes(h).  Synchronises `stream`. */
mc_status mc_estimate_uniform_noalloc(const mc_tables *t, int h, uint64_t seed, uint64_t first_index,
                                      int64_t samples, double *est, uint64_t *hits, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of requests over device-resident tables      */
/* ------------------------------------------------------------------------ */
/* A server keeps built tables on the device and runs sample and estimate
 * requests on a pool of `slots` workers, each with its own CUDA stream.
 * Requests queue in arrival order; the first queued request starts as soon
 * as a worker is idle and the device bytes it will allocate (outputs,
 * scratch, and the root or star indices it creates; for AGS a root index per
 * treelet shape and one batch of class ids) fit the device's free memory at
 * that moment on top of what the running requests were charged, and, when
 * `memory_budget` is not 0, fit that cap next to them.  With no request
 * running the head is admitted regardless (if it does not fit the device it
 * fails alone with MC_E_NOMEM).  Requests that arrive while others run are admitted as
 * workers and memory free up, and their work overlaps on the device.  A
 * request's result depends only on the tables, its seed and its sample
 * indices: it is the same alone and in any mix.  The tables must outlive the
 * server; tables built without an allocator use stream-ordered memory for
 * their per-call scratch, so workers never synchronise the device to
 * allocate. */
typedef struct mc_server mc_server;

#define MC_REQ_SAMPLE 0
#define MC_REQ_ESTIMATE 1

typedef struct {
    int kind;                  /* MC_REQ_SAMPLE or MC_REQ_ESTIMATE */
    int table;                 /* index into the server's tables */
    int h;                     /* sample requests: treelet size */
    int32_t unrooted_shape;    /* sample requests: -1 for all shapes */
    int64_t node_lo, node_hi;  /* sample requests: root range (node_hi <= 0: all nodes) */
    uint64_t seed, first_index;
    int64_t count;             /* sample requests: number of samples */
    mc_estimate_params est;    /* estimate requests */
} mc_request;

mc_status mc_server_create(const mc_tables *const *tables, int n_tables, int slots, size_t memory_budget,
                           mc_server **out);
/* Queue a request (returns at once); *id identifies it. */
mc_status mc_server_submit(mc_server *server, const mc_request *request, int64_t *id);
/* Wait for request `id` and copy its results to host buffers (any may be
 * NULL): sample requests fill nodes[count*h] (each sample's nodes ascending)
 * and classes[count]; estimate requests fill est[N_h] and hits[N_h].
 * queue_us: submit to start; latency_us: submit to completion.  A request's
 * results are delivered once. */
mc_status mc_server_wait(mc_server *server, int64_t id, uint32_t *nodes, int32_t *classes, double *est,
                         uint64_t *hits, double *queue_us, double *latency_us);
/* Stop the workers after their current requests and free the server.
 * Requests still queued are dropped; no thread may be waiting in
 * mc_server_wait on this server (its wait would never end). */
void mc_server_free(mc_server *server);

/* ------------------------------------------------------------------------ */
/* Catalogue (computed on the current device on first use, then cached)      */
/* ------------------------------------------------------------------------ */
int mc_num_shapes(int h);          /* rooted treelet shapes on h nodes */
int mc_num_unrooted(int h);        /* unrooted treelet shapes on h nodes */
int mc_num_classes(int h);         /* connected h-node graphs; -1 on error */
/* Rooted shapes of size h in id order: s_T as an integer of 2(h-1) bits
 * (DFS from the root, 1 = away from the root, children in decreasing
 * lexicographic order, Section 3.2.1), its unrooted shape id, beta_T and the
 * ids of T' and T'' (-1 for h = 1).  Host arrays of mc_num_shapes(h). */
mc_status mc_shape_info(int h, uint32_t *code, int32_t *unrooted, int32_t *beta, int32_t *left,
                        int32_t *right);
/* The level-k decompositions of round skipping (MC_BUILD_SKIP_ROUND,
 * Section 3.3.2), 4 <= k <= 8: per rooted k-shape (id order), beta_T and the
 * sizes and ids of T' and T'' of its balanced decomposition, or -1 for the
 * shapes that are not counted (host arrays of mc_num_shapes(k)); and per
 * unrooted k-shape, a_j, the rooted copies the level-k table holds for each
 * copy (host array of mc_num_unrooted(k); 0 for the star).  Any array may be
 * NULL. */
mc_status mc_skip_round_info(int k, int32_t *beta, int32_t *left_size, int32_t *left,
                             int32_t *right_size, int32_t *right, int32_t *copies);
/* Canonical adjacency words of the connected h-node graphs, ascending (host
 * uint32[mc_num_classes(h)]).  Word of a labelled graph: pairs (i, j), i < j,
 * in lexicographic order, the first pair in the most significant of the
 * C(h,2) bits; canonical word: the smallest over all relabelings. */
mc_status mc_class_codes(int h, uint32_t *codes);
/* sigma_i (spanning trees of class i) and sigma_ij (those isomorphic to
 * unrooted shape j), host int64[N_h] and int64[N_h * mc_num_unrooted(h)]. */
mc_status mc_sigma(int h, int64_t *sigma_i, int64_t *sigma_ij);

/* ------------------------------------------------------------------------ */
/* Tracing                                                                   */
/* ------------------------------------------------------------------------ */
/* on = 1: every kernel the library launches is bracketed by CUDA events
 * recorded on its own stream.  on = 3: the same, and sampler launches that
 * fill the GPU (dense tables) count the bytes they read and write -- under
 * "sample" the bytes of the data items, under "sample sectors" the same
 * accesses at 32 bytes per random access (contiguous runs by their bytes) --
 * in an instantiation of their own that synchronises its stream after each
 * launch (so on = 1 times the uncounted kernel).  on = 0: off.
 * mc_profile_read synchronises the events and reports, per kernel name, the
 * summed device time (ms), the number of launches and the counted bytes (0
 * where nothing is counted): names are written NUL-separated
 * into `names`, at most `max` kernels, their number into *count; any output
 * array may be NULL.  mc_launch_count is the number of kernels launched since
 * the library was loaded, whether or not profiling is on.  Profiling state is
 * process-wide. */
mc_status mc_profile_enable(int on);
mc_status mc_profile_reset(void);
mc_status mc_profile_read(char *names, size_t names_bytes, double *ms, int64_t *launches, int64_t *bytes,
                          int max, int *count);
int64_t mc_launch_count(void);

const char *mc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MOTIF_H */
