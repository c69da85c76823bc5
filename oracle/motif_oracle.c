/*
 * motif_oracle.c -- plain CPU oracle for colour-coding treelet counting,
 * uniform and adaptive graphlet sampling (Bressan, Leucci, Panconesi,
 * "Faster motif counting via succinct color coding and adaptive sampling").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the treelet catalogue is
 * passed in by the Python side of the oracle (oracle/catalog.py).
 *
 * All counts are exact: unsigned __int128 with checked additions and
 * multiplications.  In 64-bit mode the same values are computed and any
 * stored count, neighbour sum or merge numerator >= 2^64 is reported as an
 * overflow.  Floating point appears only in the estimators, with the order
 * of operations written out; build with -ffp-contract=off.
 *
 * Parallelism: the build loops over nodes with a plain thread pool, one
 * node per task, as the paper's build does (Section 3.4.3).  Nothing else
 * is reordered, blocked or fused beyond the formulas cited at each step.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

enum { OC_OK = 0, OC_INVALID = 1, OC_NOMEM = 2, OC_OVERFLOW = 3, OC_INTERNAL = 7 };

#define MAXK 8

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies with  */
/* a Weyl-sequence key schedule.                                            */
/* ------------------------------------------------------------------------ */
void oc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Colouring (Section 2.1): c_v uniform in [k].  Counter (v, 0, 0, 0xC010),
 * key = seed; c_v = floor(k * x0 / 2^32) of the first output word. */
void oc_color(int64_t n, int k, uint64_t seed, uint8_t *colors)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int64_t v = 0; v < n; ++v) {
        uint32_t ctr[4] = { (uint32_t)v, 0u, 0u, 0xC010u }, x[4];
        oc_philox4x32_10(ctr, key, x);
        colors[v] = (uint8_t)(((uint64_t)x[0] * (uint64_t)k) >> 32);
    }
}

/* Biased colouring (Section 3.5): colours 1..k-1 each with probability
 * lambda = L / 2^32, colour 0 with 1 - (k-1) lambda; (k-1) L <= 2^32.  The
 * same counter as above; x = x0: colour 1 + floor(x / L) when x < (k-1) L,
 * else 0.  L = 0 is the uniform colouring above. */
int oc_color_biased(int64_t n, int k, uint64_t seed, uint32_t L, uint8_t *colors)
{
    if (L == 0) { oc_color(n, k, seed, colors); return OC_OK; }
    if ((uint64_t)(k - 1) * L > 4294967296ull) return OC_INVALID;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    const uint64_t rare = (uint64_t)(k - 1) * L;
    for (int64_t v = 0; v < n; ++v) {
        uint32_t ctr[4] = { (uint32_t)v, 0u, 0u, 0xC010u }, x[4];
        oc_philox4x32_10(ctr, key, x);
        colors[v] = (uint8_t)((uint64_t)x[0] < rare ? 1u + x[0] / L : 0u);
    }
    return OC_OK;
}

/* uniform(W), W >= 1: 128 bits from Philox with counter
 * (index_lo, index_hi, step, attempt), masked to the smallest power of two
 * >= W, accepted when < W, else attempt + 1. */
static u128 draw_below(uint64_t seed, uint64_t index, uint32_t step, u128 W)
{
    if (W == 0) abort();   /* a weight of zero here is a broken table */
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    int bits = 0;
    u128 wm1 = W - 1;
    while (bits < 128 && (wm1 >> bits) != 0) ++bits;
    u128 mask = bits == 128 ? ~(u128)0 : (((u128)1 << bits) - 1);
    for (uint32_t attempt = 0;; ++attempt) {
        uint32_t ctr[4] = { (uint32_t)index, (uint32_t)(index >> 32), step, attempt }, x[4];
        oc_philox4x32_10(ctr, key, x);
        u128 r = (u128)x[0] | ((u128)x[1] << 32) | ((u128)x[2] << 64) | ((u128)x[3] << 96);
        r &= mask;
        if (r < W) return r;
    }
}

void oc_draw_below(uint64_t seed, uint64_t index, uint32_t step, const uint64_t W[2], uint64_t out[2])
{
    u128 w = (u128)W[0] | ((u128)W[1] << 64);
    u128 r = draw_below(seed, index, step, w);
    out[0] = (uint64_t)r; out[1] = (uint64_t)(r >> 64);
}

/* ------------------------------------------------------------------------ */
/* Tables                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, nnz;
    int64_t *row_ptr;
    uint32_t *col;
    uint8_t *colors;
    int k, width;                 /* width: 64 or 128 */
    int zero_root;                /* level k stored at colour-0 nodes only (Section 3.4.1) */
    int skip_round;               /* level k-1 not built; level k by balanced decompositions
                                     (Section 3.3.2); shapes with left < 0 are not counted */
    int64_t copies[MAXK + 1][32]; /* per unrooted shape of size h: rooted copies per copy */
    int nshape;
    int32_t *size, *local, *left, *right, *beta, *unrooted;
    int first[MAXK + 2];          /* global id of the first shape of size h */
    int r[MAXK + 1];              /* rooted shapes of size h */
    int nsub[MAXK + 1];           /* C(k, h) */
    int mask_rank[1 << MAXK];     /* rank of a mask among masks of its popcount, ascending */
    int rank_mask[MAXK + 1][70];
    u128 *c[MAXK + 1];            /* c[h][(v * r_h + s) * C(k,h) + rank(C)] */
    int nthreads;
} oc_tables;

static inline int popc(unsigned x) { return __builtin_popcount(x); }

static inline u128 *cell(const oc_tables *t, int h, int64_t v, int s_local, unsigned mask)
{
    return &t->c[h][((size_t)v * t->r[h] + s_local) * t->nsub[h] + t->mask_rank[mask]];
}

static inline u128 count_of(const oc_tables *t, int g, unsigned mask, int64_t v)
{
    /* c(T_C, v) for global shape g; zero unless |C| = |T| */
    int h = t->size[g];
    if (popc(mask) != h) return 0;
    return *cell(t, h, v, t->local[g], mask);
}

void oc_free(oc_tables *t)
{
    if (!t) return;
    for (int h = 0; h <= MAXK; ++h) free(t->c[h]);
    free(t->row_ptr); free(t->col); free(t->colors);
    free(t->size); free(t->local); free(t->left); free(t->right); free(t->beta); free(t->unrooted);
    free(t);
}

static int32_t *dup32(const int32_t *src, int n)
{
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (p && n > 0) memcpy(p, src, sizeof(int32_t) * (size_t)n);
    return p;
}

/* ---- build, Eq. (1) ----------------------------------------------------- */
typedef struct {
    oc_tables *t;
    int h;
    int tid;
    int status;
} build_job;

static int too_wide(const oc_tables *t, u128 x)
{
    return t->width == 64 && (x >> 64) != 0;
}

/* c(T_C, v) = (1/beta_T) sum_{u ~ v} sum_{C' subset C, |C'| = |T'|} c(T'_C', v) c(T''_{C \ C'}, u),
 * for every shape T of size h and every colour set C of size h containing c_v
 * (other sets have count 0 at v).  Written literally: u outer, C' inner. */
static void *build_level_worker(void *arg)
{
    build_job *job = (build_job *)arg;
    oc_tables *t = job->t;
    const int h = job->h;
    for (int64_t v = job->tid; v < t->n; v += t->nthreads) {
        const unsigned cv = 1u << t->colors[v];
        /* Zero-rooting (Section 3.4.1): level-k counts are kept only at nodes
         * of colour 0; every colourful k-treelet has exactly one such node. */
        if (t->zero_root && h == t->k && t->colors[v] != 0) continue;
        for (int g = t->first[h]; g < t->first[h + 1]; ++g) {
            const int a = t->left[g], b = t->right[g];
            if (a < 0) continue;                 /* not counted (round skipping) */
            const int ha = t->size[a];
            for (int q = 0; q < t->nsub[h]; ++q) {          /* |C| = h, c_v in C */
                const unsigned C = (unsigned)t->rank_mask[h][q];
                if (!(C & cv)) continue;
                u128 num = 0;
                for (int64_t e = t->row_ptr[v]; e < t->row_ptr[v + 1]; ++e) {
                    const int64_t u = t->col[e];
                    for (int q1 = 0; q1 < t->nsub[ha]; ++q1) {   /* C' subset C, |C'| = |T'|, c_v in C' */
                        const unsigned C1 = (unsigned)t->rank_mask[ha][q1];
                        if ((C1 & ~C) || !(C1 & cv)) continue;
                        const u128 x = count_of(t, a, C1, v);
                        const u128 y = count_of(t, b, C & ~C1, u);
                        u128 p;
                        if (__builtin_mul_overflow(x, y, &p) || __builtin_add_overflow(num, p, &num)) {
                            job->status = OC_OVERFLOW;
                            return NULL;
                        }
                    }
                }
                if (too_wide(t, num)) { job->status = OC_OVERFLOW; return NULL; }
                if (num % (u128)t->beta[g] != 0) { job->status = OC_INTERNAL; return NULL; }
                *cell(t, h, v, t->local[g], C) = num / (u128)t->beta[g];
            }
        }
    }
    return NULL;
}

/* Neighbour sums S(T'', C'', v) = sum_{u ~ v} c(T''_{C''}, u) for every shape of
 * size h <= k-1 and every C'' of size h without c_v.  The build above uses
 * them implicitly; this pass only checks that each fits the count width. */
static void *check_sums_worker(void *arg)
{
    build_job *job = (build_job *)arg;
    oc_tables *t = job->t;
    const int h = job->h;
    for (int64_t v = job->tid; v < t->n; v += t->nthreads) {
        const unsigned cv = 1u << t->colors[v];
        for (int g = t->first[h]; g < t->first[h + 1]; ++g)
            for (int q = 0; q < t->nsub[h]; ++q) {
                const unsigned C = (unsigned)t->rank_mask[h][q];
                if (C & cv) continue;
                u128 s = 0;
                for (int64_t e = t->row_ptr[v]; e < t->row_ptr[v + 1]; ++e)
                    if (__builtin_add_overflow(s, count_of(t, g, C, t->col[e]), &s)) {
                        job->status = OC_OVERFLOW; return NULL;
                    }
                if (too_wide(t, s)) { job->status = OC_OVERFLOW; return NULL; }
            }
    }
    return NULL;
}

static int run_pool(oc_tables *t, int h, void *(*fn)(void *))
{
    int nt = t->nthreads;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    build_job *jobs = (build_job *)calloc((size_t)nt, sizeof(build_job));
    if (!th || !jobs) { free(th); free(jobs); return OC_NOMEM; }
    for (int i = 0; i < nt; ++i) {
        jobs[i].t = t; jobs[i].h = h; jobs[i].tid = i; jobs[i].status = OC_OK;
        if (nt == 1) fn(&jobs[i]);
        else pthread_create(&th[i], NULL, fn, &jobs[i]);
    }
    int st = OC_OK;
    for (int i = 0; i < nt; ++i) {
        if (nt > 1) pthread_join(th[i], NULL);
        if (jobs[i].status != OC_OK && st == OC_OK) st = jobs[i].status;
    }
    free(th); free(jobs);
    return st;
}

static int binom(int n, int r)
{
    if (r < 0 || r > n) return 0;
    int out = 1;
    for (int i = 1; i <= r; ++i) out = out * (n - r + i) / i;
    return out;
}

/* Build all tables c(T_C, v) for |T| = 1..k.  The catalogue arrays run over
 * global shape ids (sizes 1..k, shape-id order within a size). */
oc_tables *oc_build(int64_t n, const int64_t *row_ptr, const uint32_t *col, const uint8_t *colors,
                    int k, int width, int nshape, const int32_t *size, const int32_t *local,
                    const int32_t *left, const int32_t *right, const int32_t *beta,
                    const int32_t *unrooted, const int32_t *copies, int nthreads, int zero_root,
                    int skip_round, int *status)
{
    *status = OC_INVALID;
    if (k < 1 || k > MAXK || (width != 64 && width != 128) || n < 0) return NULL;
    if (skip_round && (k < 4 || zero_root)) return NULL;
    oc_tables *t = (oc_tables *)calloc(1, sizeof(oc_tables));
    if (!t) { *status = OC_NOMEM; return NULL; }
    t->n = n; t->k = k; t->width = width; t->nshape = nshape; t->zero_root = zero_root != 0;
    t->skip_round = skip_round != 0;
    t->nthreads = nthreads < 1 ? 1 : nthreads;
    t->nnz = row_ptr[n];
    t->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    t->col = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(t->nnz > 0 ? t->nnz : 1));
    t->colors = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    t->size = dup32(size, nshape); t->local = dup32(local, nshape);
    t->left = dup32(left, nshape); t->right = dup32(right, nshape);
    t->beta = dup32(beta, nshape); t->unrooted = dup32(unrooted, nshape);
    if (!t->row_ptr || !t->col || !t->colors) { oc_free(t); *status = OC_NOMEM; return NULL; }
    memcpy(t->row_ptr, row_ptr, sizeof(int64_t) * (size_t)(n + 1));
    if (t->nnz) memcpy(t->col, col, sizeof(uint32_t) * (size_t)t->nnz);
    if (n) memcpy(t->colors, colors, (size_t)n);
    for (int64_t v = 0; v < n; ++v)
        if (t->colors[v] >= k) { oc_free(t); return NULL; }

    for (int h = 1; h <= k; ++h) { t->r[h] = 0; t->nsub[h] = binom(k, h); }
    for (int g = 0; g < nshape; ++g) t->r[size[g]]++;
    int acc = 0;
    for (int h = 1; h <= k + 1; ++h) { t->first[h] = acc; if (h <= k) acc += t->r[h]; }
    /* copies[] lists, size after size, the rooted copies per copy of every
     * unrooted shape (h, or a_j at a round-skipped level k) */
    for (int h = 1, p = 0; h <= k; ++h) {
        int nu = 0;
        for (int g = t->first[h]; g < t->first[h + 1]; ++g) if (unrooted[g] + 1 > nu) nu = unrooted[g] + 1;
        if (nu > 32) { oc_free(t); return NULL; }
        for (int j = 0; j < nu; ++j) t->copies[h][j] = copies[p++];
    }
    int cnt[MAXK + 1] = { 0 };
    for (unsigned m = 0; m < (1u << k); ++m) {       /* masks ascending */
        int p = popc(m);
        t->mask_rank[m] = cnt[p];
        t->rank_mask[p][cnt[p]++] = (int)m;
    }
    for (int h = 1; h <= k; ++h) {
        size_t cells = (size_t)n * (size_t)t->r[h] * (size_t)t->nsub[h];
        t->c[h] = (u128 *)calloc(cells ? cells : 1, sizeof(u128));
        if (!t->c[h]) { oc_free(t); *status = OC_NOMEM; return NULL; }
    }
    /* Initialisation (Section 2.1): c(T_C, v) = 1 for the one-node treelet
     * with C = {c_v}; all other one-node counts are 0. */
    for (int64_t v = 0; v < n; ++v) *cell(t, 1, v, 0, 1u << t->colors[v]) = 1;

    int st = OC_OK;
    for (int h = 2; h <= k && st == OC_OK; ++h)
        if (!(t->skip_round && h == k - 1)) st = run_pool(t, h, build_level_worker);
    for (int h = 1; h <= k - 1 && st == OC_OK; ++h)
        if (!(t->skip_round && h == k - 1)) st = run_pool(t, h, check_sums_worker);
    *status = st;
    if (st != OC_OK) { oc_free(t); return NULL; }
    return t;
}

/* Level-h table in the layout [v][shape][rank of C among size-h masks],
 * each count as two uint64 words (low, high). */
static int level_missing(const oc_tables *t, int h)
{
    return h < 1 || h > t->k || (t->skip_round && h == t->k - 1);
}

int oc_read_level(const oc_tables *t, int h, uint64_t *out)
{
    if (level_missing(t, h)) return OC_INVALID;
    size_t cells = (size_t)t->n * (size_t)t->r[h] * (size_t)t->nsub[h];
    for (size_t i = 0; i < cells; ++i) {
        out[2 * i] = (uint64_t)t->c[h][i];
        out[2 * i + 1] = (uint64_t)(t->c[h][i] >> 64);
    }
    return OC_OK;
}

/* S(T, C, v) = sum_{u ~ v} c(T_C, u) for one node, all shapes of size h and
 * all size-h masks, in the same layout as oc_read_level (one node's block). */
int oc_neighbor_sum(const oc_tables *t, int h, int64_t v, uint64_t *out)
{
    if (level_missing(t, h) || v < 0 || v >= t->n) return OC_INVALID;
    for (int s = 0; s < t->r[h]; ++s)
        for (int q = 0; q < t->nsub[h]; ++q) {
            unsigned C = (unsigned)t->rank_mask[h][q];
            u128 acc = 0;
            for (int64_t e = t->row_ptr[v]; e < t->row_ptr[v + 1]; ++e)
                acc += *cell(t, h, t->col[e], s, C);
            size_t i = (size_t)s * t->nsub[h] + q;
            out[2 * i] = (uint64_t)acc;
            out[2 * i + 1] = (uint64_t)(acc >> 64);
        }
    return OC_OK;
}

/* ---- totals (Section 2.2: t is known from the table) --------------------- */
static int shape_allowed(const oc_tables *t, int g, int h, int unrooted)
{
    return t->size[g] == h && (unrooted < 0 || t->unrooted[g] == unrooted);
}

static u128 node_total(const oc_tables *t, int h, int unrooted, int64_t v)
{
    u128 s = 0;
    for (int g = t->first[h]; g < t->first[h + 1]; ++g) {
        if (!shape_allowed(t, g, h, unrooted)) continue;
        for (int q = 0; q < t->nsub[h]; ++q) s += *cell(t, h, v, t->local[g], (unsigned)t->rank_mask[h][q]);
    }
    return s;
}

/* Rooted total R = sum_v sum_{T, C} c(T_C, v) over the shapes of size h (all,
 * or the rootings of one unrooted shape); the unrooted count of shape j is
 * R_j / h, each copy having h rootings -- or R_j itself for a zero-rooted
 * level k, where each copy is stored once, at its colour-0 node, or R_j / a_j
 * for a round-skipped level k, where a copy is stored once per node at
 * which its rooting has a balanced decomposition (the star: 0, not counted).
 * With all shapes, the unrooted count is the sum over j. */
static int shape_total(const oc_tables *t, int h, int unrooted, u128 *R, u128 *U)
{
    u128 r = 0;
    for (int64_t v = 0; v < t->n; ++v)
        if (__builtin_add_overflow(r, node_total(t, h, unrooted, v), &r)) return OC_OVERFLOW;
    u128 div = (t->zero_root && h == t->k) ? 1 : (u128)t->copies[h][unrooted];
    if (div == 0) {                       /* not counted */
        if (r != 0) return OC_INTERNAL;
        div = 1;
    }
    if (r % div != 0) return OC_INTERNAL;
    *R = r;
    *U = r / div;
    return OC_OK;
}

int oc_total(const oc_tables *t, int h, int unrooted, uint64_t rooted[2], uint64_t unrooted_count[2])
{
    if (level_missing(t, h)) return OC_INVALID;
    u128 R = 0, U = 0;
    int nu = 0;
    for (int g = t->first[h]; g < t->first[h + 1]; ++g) if (t->unrooted[g] + 1 > nu) nu = t->unrooted[g] + 1;
    for (int j = 0; j < nu; ++j) {
        if (unrooted >= 0 && j != unrooted) continue;
        u128 r, u;
        int st = shape_total(t, h, j, &r, &u);
        if (st != OC_OK) return st;
        if (__builtin_add_overflow(R, r, &R) || __builtin_add_overflow(U, u, &U)) return OC_OVERFLOW;
    }
    rooted[0] = (uint64_t)R; rooted[1] = (uint64_t)(R >> 64);
    unrooted_count[0] = (uint64_t)U; unrooted_count[1] = (uint64_t)(U >> 64);
    return OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sampling (Section 2.2)                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int h, unrooted;
    u128 *prefix;     /* inclusive prefix over v of the node totals */
    u128 R;
} root_index;

static int make_root_index(const oc_tables *t, int h, int unrooted, root_index *ri)
{
    ri->h = h; ri->unrooted = unrooted;
    ri->prefix = (u128 *)malloc(sizeof(u128) * (size_t)(t->n > 0 ? t->n : 1));
    if (!ri->prefix) return OC_NOMEM;
    u128 acc = 0;
    for (int64_t v = 0; v < t->n; ++v) {
        if (__builtin_add_overflow(acc, node_total(t, h, unrooted, v), &acc)) { free(ri->prefix); return OC_OVERFLOW; }
        ri->prefix[v] = acc;
    }
    ri->R = acc;
    return OC_OK;
}

static int is_adjacent(const oc_tables *t, int64_t a, int64_t b)
{
    int64_t lo = t->row_ptr[a], hi = t->row_ptr[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (t->col[mid] < (uint64_t)b) lo = mid + 1; else hi = mid;
    }
    return lo < t->row_ptr[a + 1] && t->col[lo] == (uint32_t)b;
}

typedef struct { int g; unsigned C; int64_t v; } dnode;

/* One colourful h-treelet, drawn uniformly among the copies whose rooted
 * shape is allowed (all shapes, or the rootings of one unrooted shape):
 *  - step 0: X = uniform(R); v = first node whose inclusive prefix exceeds X;
 *    then (T, C) = first entry of v, in (shape id, mask) ascending order,
 *    whose running sum exceeds the remainder;
 *  - then every decomposition node (T, C, v), in pre-order (T' before T''),
 *    takes the next step number: Y = uniform(beta_T c(T_C, v)); (C'', u) is
 *    the first pair, C'' over the |T''|-subsets of C \ {c_v} by ascending
 *    mask and u over N(v) ascending, at which the running sum of
 *    c(T'_{C \ C''}, v) c(T''_{C''}, u) exceeds Y;
 *  - the sample is the set of leaf nodes of the decomposition. */
static int sample_one(const oc_tables *t, const root_index *ri, uint64_t seed, uint64_t index,
                      uint32_t *nodes_out, uint32_t *root_out, int32_t *shape_out)
{
    const int h = ri->h;
    if (ri->R == 0) return OC_INVALID;
    u128 X = draw_below(seed, index, 0, ri->R);
    int64_t lo = 0, hi = t->n - 1;
    while (lo < hi) {                      /* first v with prefix[v] > X */
        int64_t mid = lo + (hi - lo) / 2;
        if (ri->prefix[mid] > X) hi = mid; else lo = mid + 1;
    }
    int64_t v = lo;
    u128 rem = X - (ri->prefix[v] - node_total(t, h, ri->unrooted, v));
    int g0 = -1; unsigned C0 = 0;
    u128 run = 0;
    for (int g = t->first[h]; g < t->first[h + 1] && g0 < 0; ++g) {
        if (!shape_allowed(t, g, h, ri->unrooted)) continue;
        for (unsigned C = 0; C < (1u << t->k); ++C) {
            if (popc(C) != h) continue;
            run += *cell(t, h, v, t->local[g], C);
            if (run > rem) { g0 = g; C0 = C; break; }
        }
    }
    if (g0 < 0) return OC_INTERNAL;
    *root_out = (uint32_t)v;
    *shape_out = t->local[g0];

    dnode stack[2 * MAXK];
    int sp = 0, nn = 0;
    uint32_t step = 0;
    stack[sp++] = (dnode){ g0, C0, v };
    while (sp > 0) {
        dnode d = stack[--sp];
        if (t->size[d.g] == 1) { nodes_out[nn++] = (uint32_t)d.v; continue; }
        ++step;
        const int a = t->left[d.g], b = t->right[d.g];
        const int hb = t->size[b];
        const unsigned cv = 1u << t->colors[d.v];
        const u128 W = (u128)t->beta[d.g] * count_of(t, d.g, d.C, d.v);
        const u128 Y = draw_below(seed, index, step, W);
        u128 acc = 0;
        int found = 0;
        unsigned rest = d.C & ~cv;
        for (unsigned C2 = 1; C2 < (1u << t->k) && !found; ++C2) {
            if ((C2 & ~rest) || popc(C2) != hb) continue;
            const u128 x = count_of(t, a, d.C & ~C2, d.v);
            for (int64_t e = t->row_ptr[d.v]; e < t->row_ptr[d.v + 1]; ++e) {
                const int64_t u = t->col[e];
                acc += x * count_of(t, b, C2, u);
                if (acc > Y) {
                    stack[sp++] = (dnode){ b, C2, u };
                    stack[sp++] = (dnode){ a, d.C & ~C2, d.v };
                    found = 1;
                    break;
                }
            }
        }
        if (!found) return OC_INTERNAL;
    }
    if (nn != h) return OC_INTERNAL;
    for (int i = 1; i < nn; ++i)            /* sort ascending */
        for (int j = i; j > 0 && nodes_out[j - 1] > nodes_out[j]; --j) {
            uint32_t tmp = nodes_out[j]; nodes_out[j] = nodes_out[j - 1]; nodes_out[j - 1] = tmp;
        }
    for (int i = 1; i < nn; ++i) if (nodes_out[i] == nodes_out[i - 1]) return OC_INTERNAL;
    return OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Graphlet classes (Section 4.4.3)                                          */
/* Adjacency word: the pairs (i, j), i < j, of the h labels in lexicographic */
/* order, first pair in the most significant of the C(h,2) bits.  Canonical  */
/* code: the smallest word over all h! relabelings.  Class id: rank of the   */
/* canonical code among those of all connected h-node graphs, ascending.     */
/* ------------------------------------------------------------------------ */
static int pair_bit(int h, int i, int j)
{
    /* position counted from the most significant end */
    int p = 0;
    for (int a = 0; a < i; ++a) p += h - 1 - a;
    p += j - i - 1;
    return binom(h, 2) - 1 - p;
}

static int word_has_edge(uint32_t w, int h, int i, int j)
{
    if (i > j) { int x = i; i = j; j = x; }
    return (w >> pair_bit(h, i, j)) & 1u;
}

static int connected_word(uint32_t w, int h)
{
    unsigned seen = 1u, frontier = 1u;
    while (frontier) {
        unsigned next = 0;
        for (int i = 0; i < h; ++i) {
            if (!(frontier >> i & 1u)) continue;
            for (int j = 0; j < h; ++j)
                if (j != i && word_has_edge(w, h, i, j) && !(seen >> j & 1u)) next |= 1u << j;
        }
        seen |= next;
        frontier = next;
    }
    return seen == (1u << h) - 1u;
}

/* permutations of [h] in lexicographic order */
static int next_perm(int *p, int h)
{
    int i = h - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return 0;
    int j = h - 1;
    while (p[j] <= p[i]) --j;
    int x = p[i]; p[i] = p[j]; p[j] = x;
    for (int a = i + 1, b = h - 1; a < b; ++a, --b) { x = p[a]; p[a] = p[b]; p[b] = x; }
    return 1;
}

/* The graph with new label i carried by old label p[i]. */
static uint32_t relabel_word(uint32_t w, int h, const int *p)
{
    uint32_t out = 0;
    for (int i = 0; i < h; ++i)
        for (int j = i + 1; j < h; ++j)
            if (word_has_edge(w, h, p[i], p[j])) out |= 1u << pair_bit(h, i, j);
    return out;
}

/* The smallest relabelled word over all h! permutations.  The adjacency
 * matrix of w and the bit position of every pair are read out once, so each
 * permutation costs one table lookup per pair (the same minimum as taking
 * relabel_word for every permutation). */
uint32_t oc_canonical_code(int h, uint32_t w)
{
    int p[MAXK], bit[MAXK][MAXK], adj[MAXK][MAXK];
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) {
            bit[i][j] = i < j ? pair_bit(h, i, j) : 0;
            adj[i][j] = i != j && word_has_edge(w, h, i, j);
        }
    for (int i = 0; i < h; ++i) p[i] = i;
    uint32_t best = w;
    do {
        uint32_t x = 0;
        for (int i = 0; i < h; ++i)
            for (int j = i + 1; j < h; ++j)
                if (adj[p[i]][p[j]]) x |= 1u << bit[i][j];
        if (x < best) best = x;
    } while (next_perm(p, h));
    return best;
}

static uint32_t *class_codes[MAXK + 1];
static int class_count[MAXK + 1];

/* Orbit sweep: scanning the words in ascending order, the first word met of
 * each isomorphism orbit is that orbit's minimum, i.e. its canonical code.
 * Bit lists per permutation make the relabelling loop touch only edges. */
static int ensure_classes(int h)
{
    if (h < 1 || h > MAXK) return OC_INVALID;
    if (class_codes[h]) return OC_OK;
    const int P = binom(h, 2);
    const uint64_t nw = (uint64_t)1 << P;
    uint8_t *seen = (uint8_t *)calloc((size_t)(nw / 8 + 1), 1);
    int nperm = 1;
    for (int i = 2; i <= h; ++i) nperm *= i;
    uint8_t *dst = (uint8_t *)malloc((size_t)nperm * (size_t)(P > 0 ? P : 1));
    uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * 16384);
    if (!seen || !dst || !codes) { free(seen); free(dst); free(codes); return OC_NOMEM; }
    /* dst[perm][bit of (i,j)] = bit of (q(i), q(j)) where q is the inverse of p */
    int p[MAXK], q[MAXK];
    for (int i = 0; i < h; ++i) p[i] = i;
    int pi = 0;
    do {
        for (int i = 0; i < h; ++i) q[p[i]] = i;
        for (int i = 0; i < h; ++i)
            for (int j = i + 1; j < h; ++j) {
                int a = q[i], b = q[j];
                if (a > b) { int x = a; a = b; b = x; }
                dst[(size_t)pi * P + pair_bit(h, i, j)] = (uint8_t)pair_bit(h, a, b);
            }
        ++pi;
    } while (next_perm(p, h));
    int nc = 0;
    for (uint64_t w = 0; w < nw; ++w) {
        if (seen[w >> 3] >> (w & 7) & 1u) continue;
        for (int m = 0; m < nperm; ++m) {
            uint32_t x = 0;
            for (uint32_t bits = (uint32_t)w; bits; bits &= bits - 1)
                x |= 1u << dst[(size_t)m * P + __builtin_ctz(bits)];
            seen[x >> 3] |= (uint8_t)(1u << (x & 7));
        }
        if (connected_word((uint32_t)w, h)) {
            if (nc >= 16384) { free(seen); free(dst); free(codes); return OC_INTERNAL; }
            codes[nc++] = (uint32_t)w;
        }
    }
    free(seen); free(dst);
    class_codes[h] = codes;
    class_count[h] = nc;
    return OC_OK;
}

int oc_num_classes(int h)
{
    if (ensure_classes(h) != OC_OK) return -1;
    return class_count[h];
}

int oc_class_codes(int h, uint32_t *out)
{
    int st = ensure_classes(h);
    if (st != OC_OK) return st;
    memcpy(out, class_codes[h], sizeof(uint32_t) * (size_t)class_count[h]);
    return OC_OK;
}

int oc_class_of_word(int h, uint32_t w)
{
    if (ensure_classes(h) != OC_OK) return -1;
    uint32_t c = oc_canonical_code(h, w);
    int lo = 0, hi = class_count[h];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (class_codes[h][mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < class_count[h] && class_codes[h][lo] == c) ? lo : -1;
}

static uint32_t induced_word(const oc_tables *t, const uint32_t *nodes, int h)
{
    uint32_t w = 0;
    for (int i = 0; i < h; ++i)
        for (int j = i + 1; j < h; ++j)
            if (is_adjacent(t, nodes[i], nodes[j])) w |= 1u << pair_bit(h, i, j);
    return w;
}

/* Draw `count` samples with indices first_index.. ; per sample: h sorted node
 * ids, the root, the rooted shape id (within size h) and the graphlet class. */
int oc_sample(const oc_tables *t, int h, int unrooted, uint64_t seed, uint64_t first_index, int64_t count,
              uint32_t *nodes, uint32_t *roots, int32_t *shapes, int32_t *classes)
{
    if (h < 2 || level_missing(t, h)) return OC_INVALID;
    int st = ensure_classes(h);
    if (st != OC_OK) return st;
    root_index ri;
    st = make_root_index(t, h, unrooted, &ri);
    if (st != OC_OK) return st;
    for (int64_t s = 0; s < count && st == OC_OK; ++s) {
        st = sample_one(t, &ri, seed, first_index + (uint64_t)s, nodes + s * h, roots + s, shapes + s);
        if (st == OC_OK) classes[s] = oc_class_of_word(h, induced_word(t, nodes + s * h, h));
    }
    free(ri.prefix);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Uncoloured star sampling (Section 3.3.2)                                  */
/* A uniform h-star of G: the centre v with probability C(d_v, h-1) / S,     */
/* S = sum_v C(d_v, h-1) (step 16: X = uniform(S), v = first node whose      */
/* inclusive prefix exceeds X), then h-1 distinct neighbours uniformly: for  */
/* t = 0..h-2, step 17 + t draws x = uniform(d_v - t) and takes the x-th     */
/* neighbour position, ascending, among those not yet taken.                */
/* ------------------------------------------------------------------------ */
#define STAR_STEP 16u

static int binom_u128(int64_t d, int r, u128 *out)
{
    /* C(d, r) = prod_{i=1..r} (d - r + i) / i, every partial product being
     * the integer C(d - r + i, i) */
    if (d < r) { *out = 0; return OC_OK; }
    u128 c = 1;
    for (int i = 1; i <= r; ++i) {
        if (__builtin_mul_overflow(c, (u128)(d - r + i), &c)) return OC_OVERFLOW;
        c /= (u128)i;
    }
    *out = c;
    return OC_OK;
}

int oc_star_total(const oc_tables *t, int h, uint64_t out[2])
{
    u128 S = 0;
    for (int64_t v = 0; v < t->n; ++v) {
        u128 c;
        if (binom_u128(t->row_ptr[v + 1] - t->row_ptr[v], h - 1, &c) != OC_OK ||
            __builtin_add_overflow(S, c, &S)) return OC_OVERFLOW;
    }
    out[0] = (uint64_t)S; out[1] = (uint64_t)(S >> 64);
    return OC_OK;
}

static int star_prefix(const oc_tables *t, int h, u128 **prefix, u128 *S)
{
    *prefix = (u128 *)malloc(sizeof(u128) * (size_t)(t->n > 0 ? t->n : 1));
    if (!*prefix) return OC_NOMEM;
    u128 acc = 0;
    for (int64_t v = 0; v < t->n; ++v) {
        u128 c;
        if (binom_u128(t->row_ptr[v + 1] - t->row_ptr[v], h - 1, &c) != OC_OK ||
            __builtin_add_overflow(acc, c, &acc)) { free(*prefix); *prefix = NULL; return OC_OVERFLOW; }
        (*prefix)[v] = acc;
    }
    *S = acc;
    return OC_OK;
}

static int star_one(const oc_tables *t, int h, const u128 *prefix, u128 S, uint64_t seed, uint64_t index,
                    uint32_t *nodes_out, uint32_t *centre_out)
{
    if (S == 0) return OC_INVALID;
    u128 X = draw_below(seed, index, STAR_STEP, S);
    int64_t lo = 0, hi = t->n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (prefix[mid] > X) hi = mid; else lo = mid + 1;
    }
    const int64_t v = lo, d = t->row_ptr[v + 1] - t->row_ptr[v];
    int64_t pos[MAXK];
    int taken = 0;
    for (int s = 0; s < h - 1; ++s) {
        int64_t x = (int64_t)draw_below(seed, index, STAR_STEP + 1u + (uint32_t)s, (u128)(d - s));
        int i = 0;
        while (i < taken && pos[i] <= x) { ++x; ++i; }    /* skip the taken positions */
        for (int j = taken; j > i; --j) pos[j] = pos[j - 1];
        pos[i] = x;
        ++taken;
    }
    nodes_out[0] = (uint32_t)v;
    for (int s = 0; s < h - 1; ++s) nodes_out[1 + s] = t->col[t->row_ptr[v] + pos[s]];
    for (int i = 1; i < h; ++i)
        for (int j = i; j > 0 && nodes_out[j - 1] > nodes_out[j]; --j) {
            uint32_t tmp = nodes_out[j]; nodes_out[j] = nodes_out[j - 1]; nodes_out[j - 1] = tmp;
        }
    *centre_out = (uint32_t)v;
    return OC_OK;
}

/* `count` uncoloured h-stars with indices first_index..: sorted nodes, the
 * centre and the graphlet class of each. */
int oc_sample_stars(const oc_tables *t, int h, uint64_t seed, uint64_t first_index, int64_t count,
                    uint32_t *nodes, uint32_t *centres, int32_t *classes)
{
    if (h < 2 || h > MAXK) return OC_INVALID;
    int st = ensure_classes(h);
    if (st != OC_OK) return st;
    u128 *prefix, S;
    st = star_prefix(t, h, &prefix, &S);
    if (st != OC_OK) return st;
    for (int64_t s = 0; s < count && st == OC_OK; ++s) {
        st = star_one(t, h, prefix, S, seed, first_index + (uint64_t)s, nodes + s * h, centres + s);
        if (st == OC_OK) classes[s] = oc_class_of_word(h, induced_word(t, nodes + s * h, h));
    }
    free(prefix);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Spanning trees (Section 4.4.3)                                            */
/* ------------------------------------------------------------------------ */

/* sigma_i by Kirchhoff's matrix-tree theorem: the determinant of the
 * Laplacian with its last row and column removed, by fraction-free
 * (Bareiss) elimination in exact integers. */
int64_t oc_spanning_trees(int h, uint32_t w)
{
    if (h == 1) return 1;
    int64_t L[MAXK][MAXK];
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) L[i][j] = 0;
    for (int i = 0; i < h; ++i)
        for (int j = i + 1; j < h; ++j)
            if (word_has_edge(w, h, i, j)) { L[i][j] = L[j][i] = -1; L[i][i]++; L[j][j]++; }
    int m = h - 1;
    int64_t prev = 1, sign = 1;
    for (int p = 0; p < m; ++p) {
        if (L[p][p] == 0) {
            int r = p + 1;
            while (r < m && L[r][p] == 0) ++r;
            if (r == m) return 0;
            for (int c = 0; c < m; ++c) { int64_t x = L[p][c]; L[p][c] = L[r][c]; L[r][c] = x; }
            sign = -sign;
        }
        for (int i = p + 1; i < m; ++i) {
            for (int j = p + 1; j < m; ++j)
                L[i][j] = (L[i][j] * L[p][p] - L[i][p] * L[p][j]) / prev;
        }
        prev = L[p][p];
    }
    return sign * L[m - 1][m - 1];
}

/* sigma_ij: the spanning trees of graphlet H_i isomorphic to the unrooted
 * treelet T_j, by the paper's recipe: run the build-up on H_i with every
 * node given its own colour; then the colourful h-treelets are all spanning
 * trees, and sum over rootings of T_j of c(T_[h], v), divided by h, counts
 * the spanning trees of shape j.  out: [n_classes][n_unrooted].  The
 * classes are independent and are spread over threads. */
typedef struct {
    int h, nshape, n_unrooted, tid, nthreads, status;
    const int32_t *size, *local, *left, *right, *beta, *unrooted, *copies;
    int64_t *out;
} sigma_job;

static void *sigma_worker(void *arg)
{
    sigma_job *jb = (sigma_job *)arg;
    const int h = jb->h;
    for (int ci = jb->tid; ci < class_count[h]; ci += jb->nthreads) {
        uint32_t w = class_codes[h][ci];
        int64_t row_ptr[MAXK + 1];
        uint32_t col[MAXK * MAXK];
        int64_t e = 0;
        for (int i = 0; i < h; ++i) {
            row_ptr[i] = e;
            for (int j = 0; j < h; ++j)
                if (j != i && word_has_edge(w, h, i, j)) col[e++] = (uint32_t)j;
        }
        row_ptr[h] = e;
        uint8_t colors[MAXK];
        for (int i = 0; i < h; ++i) colors[i] = (uint8_t)i;
        int st;
        oc_tables *t = oc_build(h, row_ptr, col, colors, h, 128, jb->nshape, jb->size, jb->local,
                                jb->left, jb->right, jb->beta, jb->unrooted, jb->copies, 1, 0, 0, &st);
        if (!t) { jb->status = st; return NULL; }
        for (int j = 0; j < jb->n_unrooted; ++j) {
            uint64_t R[2], U[2];
            st = oc_total(t, h, j, R, U);
            if (st != OC_OK) { oc_free(t); jb->status = st; return NULL; }
            jb->out[(size_t)ci * jb->n_unrooted + j] = (int64_t)U[0];
        }
        oc_free(t);
    }
    return NULL;
}

int oc_sigma_matrix(int h, int nshape, const int32_t *size, const int32_t *local, const int32_t *left,
                    const int32_t *right, const int32_t *beta, const int32_t *unrooted,
                    const int32_t *copies, int n_unrooted, int64_t *out, int nthreads)
{
    int st = ensure_classes(h);
    if (st != OC_OK) return st;
    if (nthreads < 1) nthreads = 1;
    pthread_t th[64];
    sigma_job jobs[64];
    if (nthreads > 64) nthreads = 64;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (sigma_job){ h, nshape, n_unrooted, i, nthreads, OC_OK, size, local, left, right,
                               beta, unrooted, copies, out };
        pthread_create(&th[i], NULL, sigma_worker, &jobs[i]);
    }
    for (int i = 0; i < nthreads; ++i) {
        pthread_join(th[i], NULL);
        if (jobs[i].status != OC_OK && st == OC_OK) st = jobs[i].status;
    }
    return st;
}

/* ------------------------------------------------------------------------ */
/* Estimators                                                                */
/* ------------------------------------------------------------------------ */

/* 1 / p, p = k! / ((k-h)! k^h): the probability that a fixed h-node set is
 * colourful (Section 2.2 gives p_k = k!/k^k for h = k).  Both integers are
 * exact in double; one rounding. */
static double inv_colorful_prob(int k, int h)
{
    double num = 1.0, den = 1.0;
    for (int i = 0; i < h; ++i) num *= (double)k;
    for (int i = 1; i <= k - h; ++i) num *= (double)i;
    for (int i = 1; i <= k; ++i) den *= (double)i;
    return num / den;
}

/* 1 / p under the biased colouring: an h-node set is colourful when its
 * colours are distinct, with probability h! e_h(p_0, lambda, ..., lambda) =
 * h! (C(k-1,h) lambda^h + C(k-1,h-1) lambda^(h-1) p_0), p_0 = 1 - (k-1) lambda
 * (Section 3.5 gives the leading terms j! lambda^j and j! lambda^(j-1)).
 * lambda and p_0 are exact doubles; the rest is evaluated in this order. */
static double inv_colorful_prob_biased(int k, int h, uint32_t L)
{
    if (L == 0) return inv_colorful_prob(k, h);
    const double lam = (double)L / 4294967296.0;
    const double p0 = (double)(4294967296ull - (uint64_t)(k - 1) * L) / 4294967296.0;
    double lh1 = 1.0;
    for (int i = 0; i < h - 1; ++i) lh1 *= lam;
    double fact = 1.0;
    for (int i = 2; i <= h; ++i) fact *= (double)i;
    const double p = fact * ((double)binom(k - 1, h) * (lh1 * lam) + (double)binom(k - 1, h - 1) * (lh1 * p0));
    return 1.0 / p;
}

double oc_inv_colorful_prob(int k, int h, uint32_t L) { return inv_colorful_prob_biased(k, h, L); }

static double u128_to_double(u128 x) { return (double)x; }

/* Graphlets that only stars span (sigma'_i = 0) on a round-skipped level k
 * (Section 3.3.2): n_star uncoloured h-stars, hits*_i of them spanning H_i;
 * chi-bar*_i = hits*_i / n_star estimates g_i sigma*_i / S (sigma*_i: the
 * spanning stars of H_i, S: the h-stars of G), so
 * g-hat_i = ((S * hits*_i) / (sigma*_i * n_star)), with no 1/p: the stars
 * carry no colours.  Their hits are the star hits.  With S = 0 there is no
 * star and the estimate is 0. */
static int star_estimates(const oc_tables *t, int h, uint64_t seed, uint64_t first_index, int64_t n_star,
                          const int64_t *sigma_prime, const int64_t *sigma_star, double *est, uint64_t *hits)
{
    const int ncls = class_count[h];
    u128 *prefix, S;
    int st = star_prefix(t, h, &prefix, &S);
    if (st != OC_OK) return st;
    uint64_t *sh = (uint64_t *)calloc((size_t)ncls, sizeof(uint64_t));
    if (!sh) { free(prefix); return OC_NOMEM; }
    uint32_t nodes[MAXK], centre;
    for (int64_t s = 0; S > 0 && s < n_star && st == OC_OK; ++s) {
        st = star_one(t, h, prefix, S, seed, first_index + (uint64_t)s, nodes, &centre);
        if (st != OC_OK) break;
        int cls = oc_class_of_word(h, induced_word(t, nodes, h));
        if (cls < 0) { st = OC_INTERNAL; break; }
        sh[cls]++;
    }
    free(prefix);
    if (st == OC_OK) {
        const double Sd = u128_to_double(S);
        for (int i = 0; i < ncls; ++i) {
            if (sigma_prime[i] != 0) continue;
            hits[i] = sh[i];
            est[i] = (S > 0 && n_star > 0 && sigma_star[i] > 0)
                         ? (Sd * (double)sh[i]) / ((double)sigma_star[i] * (double)n_star) : 0.0;
        }
    }
    free(sh);
    return st;
}

/* Uniform sampling estimator (Section 2.2): with N samples, hits_i of them
 * spanning graphlet H_i, chi-bar_i = hits_i / N estimates E[chi_i] =
 * c_i sigma_i / t, so c-hat_i = t (hits_i / N) / sigma_i and
 * g-hat_i = c-hat_i / p, evaluated as ((t * hits_i) / (sigma_i * N)) * (1/p).
 * On a round-skipped level k a copy of tree j is drawn with probability
 * a_j / R (R: the rooted total), so chi-bar_i estimates c_i sigma'_i / R with
 * sigma'_i = sum_j sigma_ij a_j, passed as `sigma`; then t is replaced by R,
 * the graphlets with sigma'_i = 0 get 0 here and their estimate from
 * n_star uncoloured stars (star_estimates). */
int oc_estimate_uniform(const oc_tables *t, int h, uint64_t seed, uint64_t first_index, int64_t N,
                        const int64_t *sigma, int64_t n_star, const int64_t *sigma_star, uint32_t bias,
                        double *est, uint64_t *hits)
{
    if (h < 2 || level_missing(t, h) || N <= 0) return OC_INVALID;
    int st = ensure_classes(h);
    if (st != OC_OK) return st;
    const int ncls = class_count[h];
    const int skipped = t->skip_round && h == t->k;
    uint64_t R[2], U[2];
    st = oc_total(t, h, -1, R, U);
    if (st != OC_OK) return st;
    const u128 tot = skipped ? ((u128)R[0] | ((u128)R[1] << 64)) : ((u128)U[0] | ((u128)U[1] << 64));
    for (int i = 0; i < ncls; ++i) hits[i] = 0;
    root_index ri;
    st = make_root_index(t, h, -1, &ri);
    if (st != OC_OK) return st;
    uint32_t nodes[MAXK], root;
    int32_t shape;
    for (int64_t s = 0; s < N; ++s) {
        st = sample_one(t, &ri, seed, first_index + (uint64_t)s, nodes, &root, &shape);
        if (st != OC_OK) { free(ri.prefix); return st; }
        int cls = oc_class_of_word(h, induced_word(t, nodes, h));
        if (cls < 0) { free(ri.prefix); return OC_INTERNAL; }
        hits[cls]++;
    }
    free(ri.prefix);
    const double td = u128_to_double(tot), ip = inv_colorful_prob_biased(t->k, h, bias);
    for (int i = 0; i < ncls; ++i)
        est[i] = sigma[i] > 0 ? ((td * (double)hits[i]) / ((double)sigma[i] * (double)N)) * ip : 0.0;
    if (skipped) return star_estimates(t, h, seed, first_index, n_star, sigma, sigma_star, est, hits);
    return OC_OK;
}

/* Adaptive graphlet sampling, Algorithm AGS (Section 4.1), with these
 * readings:
 *  - the first treelet is the most frequent one (largest t_j; ties to the
 *    smaller j); shapes with t_j = 0 are never chosen;
 *  - a switch happens when a graphlet becomes covered, i.e. when its sample
 *    count reaches cbar for the first time;
 *  - the weights w_i = sum_j n_j sigma_ij / t_j, with n_j the number of
 *    samples drawn with T_j so far, are evaluated at switch time and at the
 *    end (j ascending, each term (n_j sigma_ij) / t_j in double); this is the
 *    per-sample update of the algorithm summed up;
 *  - the next treelet minimises (sum_{i covered, ascending} (sigma_ij c_i) / w_i) / t_j,
 *    ties to the smaller j;
 *  - sampling stops when every graphlet is covered or after max_samples;
 *    on a round-skipped level k the graphlets that only stars span
 *    (sigma'_i = 0) are left out of this and estimated from n_star
 *    uncoloured stars (star_estimates); the star shape has t_j = 0;
 *  - every treelet has its own stream of sample indices: the n-th sample
 *    (0-based) drawn with T_j uses index first_index + j * 2^40 + n, so
 *    max_samples <= 2^40 (a reading: the paper does not say how random bits
 *    are drawn; with one stream per treelet, samples drawn ahead for a
 *    treelet stay valid whenever the algorithm comes back to it);
 *  - the result is est_i = (c_i / w_i) * (1/p), an estimate of the number
 *    of induced copies of H_i (c_i / w_i estimates its colourful copies);
 *    est_i = 0 when w_i = 0.
 * stats: [0] samples drawn, [1] switches, [2] graphlets covered, [3] the
 * first treelet (-1 if none).
 * Trace (for tests; any pointer may be NULL): for the first trace_cap
 * switches, trace_at[s] = samples drawn when switch s happened (the covering
 * sample included), trace_j[s] = the treelet chosen, and trace_w[s * ncls +
 * i] = the weight w_i it was chosen with. */
int oc_estimate_ags(const oc_tables *t, int h, uint64_t seed, uint64_t first_index, int64_t max_samples,
                    int64_t cbar, const int64_t *sigma_ij, int n_unrooted, int64_t n_star,
                    const int64_t *sigma_prime, const int64_t *sigma_star, uint32_t bias,
                    double *est, uint64_t *hits, int64_t *stats,
                    int64_t trace_cap, int32_t *trace_j, int64_t *trace_at, double *trace_w)
{
    if (h < 2 || level_missing(t, h) || max_samples < 0 || max_samples > ((int64_t)1 << 40) || cbar < 1)
        return OC_INVALID;
    int st = ensure_classes(h);
    if (st != OC_OK) return st;
    const int ncls = class_count[h];
    const int S = n_unrooted;
    u128 *tj = (u128 *)calloc((size_t)S, sizeof(u128));
    double *tjd = (double *)calloc((size_t)S, sizeof(double));
    double *w = (double *)calloc((size_t)ncls, sizeof(double));
    int64_t *nj = (int64_t *)calloc((size_t)S, sizeof(int64_t));
    uint8_t *covered = (uint8_t *)calloc((size_t)ncls, 1);
    root_index *ri = (root_index *)calloc((size_t)S, sizeof(root_index));
    if (!tj || !tjd || !w || !nj || !covered || !ri) { st = OC_NOMEM; goto done; }
    for (int j = 0; j < S; ++j) {
        uint64_t R[2], U[2];
        st = oc_total(t, h, j, R, U);
        if (st != OC_OK) goto done;
        tj[j] = (u128)U[0] | ((u128)U[1] << 64);
        tjd[j] = u128_to_double(tj[j]);
    }
    int cur = -1;
    for (int j = 0; j < S; ++j)
        if (tj[j] > 0 && (cur < 0 || tj[j] > tj[cur])) cur = j;
    stats[3] = cur;
    for (int i = 0; i < ncls; ++i) hits[i] = 0;
    int64_t drawn = 0, switches = 0, ncov = 0, target = ncls;
    if (t->skip_round && h == t->k) {      /* graphlets only stars span are left to the stars */
        target = 0;
        for (int i = 0; i < ncls; ++i) target += sigma_prime[i] > 0;
    }
    if (cur < 0) goto finish;
    uint32_t nodes[MAXK], root;
    int32_t shape;
    while (ncov < target && drawn < max_samples) {
        if (!ri[cur].prefix) { st = make_root_index(t, h, cur, &ri[cur]); if (st != OC_OK) goto done; }
        st = sample_one(t, &ri[cur], seed, first_index + ((uint64_t)cur << 40) + (uint64_t)nj[cur], nodes, &root,
                        &shape);
        if (st != OC_OK) goto done;
        nj[cur]++;
        drawn++;
        int i = oc_class_of_word(h, induced_word(t, nodes, h));
        if (i < 0) { st = OC_INTERNAL; goto done; }
        hits[i]++;
        if ((int64_t)hits[i] == cbar && !covered[i]) {
            covered[i] = 1;
            ncov++;
            switches++;
            for (int a = 0; a < ncls; ++a) {
                double acc = 0.0;
                for (int j = 0; j < S; ++j)
                    if (tj[j] > 0) acc += (double)(nj[j] * sigma_ij[(size_t)a * S + j]) / tjd[j];
                w[a] = acc;
            }
            int best = -1;
            double bestv = 0.0;
            for (int j = 0; j < S; ++j) {
                if (tj[j] == 0) continue;
                double acc = 0.0;
                for (int a = 0; a < ncls; ++a)
                    if (covered[a]) acc += ((double)sigma_ij[(size_t)a * S + j] * (double)hits[a]) / w[a];
                double val = acc / tjd[j];
                if (best < 0 || val < bestv) { best = j; bestv = val; }
            }
            cur = best;
            if (switches - 1 < trace_cap) {
                if (trace_j) trace_j[switches - 1] = cur;
                if (trace_at) trace_at[switches - 1] = drawn;
                if (trace_w)
                    for (int a = 0; a < ncls; ++a) trace_w[(size_t)(switches - 1) * ncls + a] = w[a];
            }
        }
    }
finish:
    for (int a = 0; a < ncls; ++a) {
        double acc = 0.0;
        for (int j = 0; j < S; ++j)
            if (tj[j] > 0) acc += (double)(nj[j] * sigma_ij[(size_t)a * S + j]) / tjd[j];
        w[a] = acc;
    }
    {
        const double ip = inv_colorful_prob_biased(t->k, h, bias);
        for (int a = 0; a < ncls; ++a) est[a] = w[a] > 0.0 ? ((double)hits[a] / w[a]) * ip : 0.0;
    }
    stats[0] = drawn; stats[1] = switches; stats[2] = ncov;
    st = OC_OK;
    if (t->skip_round && h == t->k)
        st = star_estimates(t, h, seed, first_index, n_star, sigma_prime, sigma_star, est, hits);
done:
    if (ri) for (int j = 0; j < S; ++j) free(ri[j].prefix);
    free(ri); free(tj); free(tjd); free(w); free(nj); free(covered);
    return st;
}

int64_t oc_n(const oc_tables *t) { return t->n; }
