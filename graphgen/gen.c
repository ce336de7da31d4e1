/*
 * Seeded synthetic graph generators (Erdos-Renyi, R-MAT, Chung-Lu) and the
 * CSR assembly they share: symmetrise, drop self-loops, sort each row and
 * remove duplicate arcs.
 *
 * This module produces INPUTS only.  It holds none of the Katz arithmetic, so
 * both the CPU oracle and the CUDA path may consume its graphs.
 *
 * Randomness is counter based: draw number t of stream s is
 * splitmix64(seed ^ stream_key(s) + t * golden), the SplitMix64 output
 * function of Steele, Lea and Flood (OOPSLA 2014).  Every edge is a pure
 * function of (seed, edge index), so the generated multiset of arcs does not
 * depend on the number of threads; CSR assembly sorts every row, so the final
 * CSR is bit-identical for any thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* draw t of stream `key` under `seed` */
static inline uint64_t draw(uint64_t seed, uint64_t key, uint64_t t) {
    return mix64(seed ^ (mix64(key) + (t + 1) * GOLDEN));
}

/* uniform double in [0,1) from the top 53 bits */
static inline double unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) by 128-bit multiply-shift (Lemire) */
static inline uint64_t below(uint64_t x, uint64_t n) {
    return (uint64_t)(((unsigned __int128)x * n) >> 64);
}

/* ------------------------------------------------------------------------- */
/* CSR assembly                                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t *rowptr;  /* n+1 */
    int32_t *col;     /* nnz */
} gg_csr;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t *p, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t v = p[i];
            int64_t j = i - 1;
            while (j >= 0 && p[j] > v) { p[j + 1] = p[j]; --j; }
            p[j + 1] = v;
        }
    } else {
        qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Build a symmetric, sorted, duplicate-free CSR from m undirected pairs
 * (u[e], v[e]).  Pairs with u == v are skipped.  Returns NULL on allocation
 * failure.
 */
static gg_csr *assemble(int64_t n, int64_t m, const int32_t *u, const int32_t *v) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] == v[e]) continue;
        __atomic_fetch_add(&cnt[u[e]], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&cnt[v[e]], 1, __ATOMIC_RELAXED);
    }
    int64_t *start = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!start) { free(cnt); return NULL; }
    start[0] = 0;
    for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + cnt[i];
    int64_t arcs = start[n];
    int32_t *tmp = (int32_t *)malloc((size_t)(arcs > 0 ? arcs : 1) * sizeof(int32_t));
    if (!tmp) { free(cnt); free(start); return NULL; }
    memcpy(cnt, start, (size_t)n * sizeof(int64_t)); /* cursors */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] == v[e]) continue;
        int64_t p = __atomic_fetch_add(&cnt[u[e]], 1, __ATOMIC_RELAXED);
        tmp[p] = v[e];
        p = __atomic_fetch_add(&cnt[v[e]], 1, __ATOMIC_RELAXED);
        tmp[p] = u[e];
    }
    /* sort + dedup every row in place; cnt[i] becomes the unique length */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int32_t *p = tmp + start[i];
        int64_t len = start[i + 1] - start[i];
        sort_row(p, len);
        int64_t w = 0;
        for (int64_t j = 0; j < len; ++j)
            if (w == 0 || p[j] != p[w - 1]) p[w++] = p[j];
        cnt[i] = w;
    }
    gg_csr *g = (gg_csr *)malloc(sizeof(gg_csr));
    g->n = n;
    g->rowptr = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) g->rowptr[i + 1] = g->rowptr[i] + cnt[i];
    g->nnz = g->rowptr[n];
    g->col = (int32_t *)malloc((size_t)(g->nnz > 0 ? g->nnz : 1) * sizeof(int32_t));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        memcpy(g->col + g->rowptr[i], tmp + start[i], (size_t)cnt[i] * sizeof(int32_t));
    free(tmp);
    free(start);
    free(cnt);
    return g;
}

/* ------------------------------------------------------------------------- */
/* public API                                                                 */
/* ------------------------------------------------------------------------- */

int64_t gg_n(const gg_csr *g) { return g->n; }
int64_t gg_nnz(const gg_csr *g) { return g->nnz; }
void gg_copy(const gg_csr *g, int64_t *rowptr, int32_t *col) {
    memcpy(rowptr, g->rowptr, ((size_t)g->n + 1) * sizeof(int64_t));
    if (g->nnz) memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
}
void gg_free(gg_csr *g) {
    if (!g) return;
    free(g->rowptr);
    free(g->col);
    free(g);
}

int gg_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Disjoint union of a given symmetric CSR (ids 0..n0-1), a band graph on
 * n_band nodes (ids n0.., i ~ j iff 0 < |i - j| <= d) and n_pad isolated
 * nodes (ids after the band).  The band's rows are sorted and duplicate-free
 * by construction; it pads a graph to an exact size (n + nnz), e.g. just below
 * the range of 32-bit row offsets.
 */
gg_csr *gg_band_union(int64_t n0, const int64_t *rowptr0, const int32_t *col0, int64_t n_band, int64_t d,
                      int64_t n_pad) {
    if (n0 < 0 || n_band < 0 || d < 0 || n_pad < 0) return NULL;
    const int64_t n = n0 + n_band + n_pad;
    gg_csr *g = (gg_csr *)malloc(sizeof(gg_csr));
    if (!g) return NULL;
    g->n = n;
    g->rowptr = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!g->rowptr) { free(g); return NULL; }
    for (int64_t i = 0; i <= n0; ++i) g->rowptr[i] = rowptr0[i];
    for (int64_t b = 0; b < n_band; ++b) {
        const int64_t lo = b - d < 0 ? 0 : b - d, hi = b + d > n_band - 1 ? n_band - 1 : b + d;
        g->rowptr[n0 + b + 1] = g->rowptr[n0 + b] + (hi - lo);
    }
    for (int64_t i = n0 + n_band; i < n; ++i) g->rowptr[i + 1] = g->rowptr[i];
    g->nnz = g->rowptr[n];
    g->col = (int32_t *)malloc((size_t)(g->nnz > 0 ? g->nnz : 1) * sizeof(int32_t));
    if (!g->col) { free(g->rowptr); free(g); return NULL; }
    if (rowptr0[n0]) memcpy(g->col, col0, (size_t)rowptr0[n0] * sizeof(int32_t));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < n_band; ++b) {
        const int64_t lo = b - d < 0 ? 0 : b - d, hi = b + d > n_band - 1 ? n_band - 1 : b + d;
        int32_t *p = g->col + g->rowptr[n0 + b];
        for (int64_t j = lo; j <= hi; ++j)
            if (j != b) *p++ = (int32_t)(n0 + j);
    }
    return g;
}

/* CSR of an arbitrary pair list (used for hand-made graphs and update tests) */
gg_csr *gg_from_pairs(int64_t n, int64_t m, const int32_t *u, const int32_t *v) {
    return assemble(n, m, u, v);
}

/*
 * Erdos-Renyi G(n, m): exactly m distinct undirected edges, drawn as uniform
 * ordered pairs; self-loops and repeats are rejected and redrawn.  Sequential
 * (the graph is small), with an open-addressing set of canonical pairs.
 */
gg_csr *gg_er(int64_t n, int64_t m, uint64_t seed) {
    if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return NULL;
    uint64_t cap = 1;
    while (cap < (uint64_t)(2 * m + 16)) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(cap * sizeof(uint64_t));
    int32_t *u = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    memset(set, 0xff, cap * sizeof(uint64_t));
    uint64_t t = 0;
    for (int64_t e = 0; e < m;) {
        uint64_t a = below(draw(seed, 1, t), (uint64_t)n);
        uint64_t b = below(draw(seed, 2, t), (uint64_t)n);
        ++t;
        if (a == b) continue;
        uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
        uint64_t key = (lo << 32) | hi;
        uint64_t h = mix64(key) & (cap - 1);
        int dup = 0;
        while (set[h] != ~0ULL) {
            if (set[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        set[h] = key;
        u[e] = (int32_t)lo;
        v[e] = (int32_t)hi;
        ++e;
    }
    gg_csr *g = assemble(n, m, u, v);
    free(set);
    free(u);
    free(v);
    return g;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): 2^scale vertices, edge_factor *
 * 2^scale generated pairs.  Each pair descends `scale` levels of the
 * recursive quadrant split with probabilities (a, b, c, 1-a-b-c); no noise,
 * no vertex permutation.  The result is symmetrised and deduplicated.
 */
gg_csr *gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed) {
    if (scale < 1 || scale > 30) return NULL;
    int64_t n = (int64_t)1 << scale;
    int64_t m = edge_factor * n;
    int32_t *u = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    if (!u || !v) { free(u); free(v); return NULL; }
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t s = 0, d = 0;
        for (int l = 0; l < scale; ++l) {
            double x = unit(draw(seed, 3, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
            uint32_t sb, db;
            if (x < a) { sb = 0; db = 0; }
            else if (x < ab) { sb = 0; db = 1; }
            else if (x < abc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        u[e] = (int32_t)s;
        v[e] = (int32_t)d;
    }
    gg_csr *g = assemble(n, m, u, v);
    free(u);
    free(v);
    return g;
}

/*
 * Chung-Lu graph with Pareto expected degrees.  Weights w_i = x_m * U^(-1/tail)
 * (pdf exponent tail+1), capped at sqrt(sum w).  `pairs` endpoint pairs are
 * drawn, each endpoint independently proportional to w (Walker/Vose alias
 * table), then symmetrised and deduplicated.
 */
gg_csr *gg_chung_lu(int64_t n, int64_t pairs, double tail, double x_m, uint64_t seed) {
    if (n < 2 || n > 2147483647LL) return NULL;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *prob = (double *)malloc((size_t)n * sizeof(double));
    int32_t *alias = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *small = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *large = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!w || !prob || !alias || !small || !large) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double x = unit(draw(seed, 4, (uint64_t)i));
        w[i] = x_m * pow(1.0 - x, -1.0 / tail);
    }
    double sum = 0.0; /* sequential: the cap must not depend on the thread count */
    for (int64_t i = 0; i < n; ++i) sum += w[i];
    const double cap = sqrt(sum);
    double csum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (w[i] > cap) w[i] = cap;
        csum += w[i];
    }
    /* Vose's alias method */
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        prob[i] = w[i] * (double)n / csum;
        if (prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns], l = large[--nl];
        alias[s] = l;
        prob[l] = (prob[l] + prob[s]) - 1.0;
        if (prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int32_t l = large[--nl]; prob[l] = 1.0; alias[l] = l; }
    while (ns > 0) { int32_t s = small[--ns]; prob[s] = 1.0; alias[s] = s; }
    free(small);
    free(large);
    free(w);
    int32_t *u = (int32_t *)malloc((size_t)pairs * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)pairs * sizeof(int32_t));
    if (!u || !v) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < pairs; ++e) {
        int32_t ends[2];
        for (int k = 0; k < 2; ++k) {
            uint64_t t = (uint64_t)e * 4u + 2u * (uint64_t)k;
            uint64_t i = below(draw(seed, 5, t), (uint64_t)n);
            double y = unit(draw(seed, 5, t + 1));
            ends[k] = (y < prob[i]) ? (int32_t)i : alias[i];
        }
        u[e] = ends[0];
        v[e] = ends[1];
    }
    free(prob);
    free(alias);
    gg_csr *g = assemble(n, pairs, u, v);
    free(u);
    free(v);
    return g;
}

/*
 * A stream of update batches for the dynamic experiments.  Given the current
 * graph (sorted CSR), draw `m` undirected updates: with probability
 * p_insert a uniform non-edge {a,b} (a != b) not already used in this batch,
 * otherwise a uniform existing edge (an arc chosen uniformly, so an edge with
 * probability 2/nnz) not already used in this batch.  Writes src, dst,
 * is_insert (1/0).  Returns the number written (== m unless the graph has no
 * edges to delete).
 */
static int has_arc(const int64_t *rowptr, const int32_t *col, int32_t a, int32_t b) {
    int64_t lo = rowptr[a], hi = rowptr[a + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < rowptr[a + 1] && col[lo] == b;
}

int64_t gg_update_batch(int64_t n, const int64_t *rowptr, const int32_t *col, int64_t m,
                        double p_insert, uint64_t seed, int32_t *src, int32_t *dst, uint8_t *is_insert) {
    int64_t nnz = rowptr[n];
    uint64_t cap = 1;
    while (cap < (uint64_t)(4 * m + 16)) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(cap * sizeof(uint64_t));
    memset(set, 0xff, cap * sizeof(uint64_t));
    uint64_t t = 0;
    int64_t e = 0;
    int64_t guard = 0;
    while (e < m && guard < 1000 * (m + 10)) {
        ++guard;
        int ins = unit(draw(seed, 6, t)) < p_insert;
        uint64_t a, b;
        if (ins) {
            a = below(draw(seed, 7, t), (uint64_t)n);
            b = below(draw(seed, 8, t), (uint64_t)n);
            ++t;
            if (a == b || has_arc(rowptr, col, (int32_t)a, (int32_t)b)) continue;
        } else {
            ++t;
            if (nnz == 0) continue;
            uint64_t arc = below(draw(seed, 9, t), (uint64_t)nnz);
            int64_t lo = 0, hi = n; /* row containing arc: last i with rowptr[i] <= arc */
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) >> 1;
                if ((uint64_t)rowptr[mid] <= arc) lo = mid; else hi = mid;
            }
            a = (uint64_t)lo;
            b = (uint64_t)col[arc];
        }
        uint64_t lo_ = a < b ? a : b, hi_ = a < b ? b : a;
        uint64_t key = (lo_ << 32) | hi_;
        uint64_t h = mix64(key) & (cap - 1);
        int dup = 0;
        while (set[h] != ~0ULL) {
            if (set[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        set[h] = key;
        src[e] = (int32_t)a;
        dst[e] = (int32_t)b;
        is_insert[e] = (uint8_t)ins;
        ++e;
    }
    free(set);
    return e;
}

/* ------------------------------------------------------------------------- */
/* Request stream for the serving workload                                    */
/* ------------------------------------------------------------------------- */
/*
 * gg_stream: `batches` update batches applied one after another to a base
 * graph (sorted symmetric CSR).  Batch j has m_j updates, m_j log-uniform in
 * [min_size, max_size]; each update is an insert with probability p_insert,
 * else a delete.  Every batch is drawn against the graph after batches
 * 0..j-1:
 *   insert: a uniform pair {a,b}, a != b, that is not an edge, not used
 *           earlier in the batch, with both degrees below deg_bound counting
 *           the batch's earlier inserts;
 *   delete: a uniform existing edge not used earlier in the batch.
 * Arrival times are a Poisson process of the given rate (exponential gaps,
 * first arrival at the first gap).
 *
 * The evolving edge set is the base CSR minus a set of deleted base edges
 * plus a list of inserted edges (with a map from edge to list slot, so an
 * inserted edge can be drawn uniformly and removed in O(1)).
 *
 * Output: offsets[batches+1] into src/dst/is_insert (capacity `cap`) and
 * arrival[batches] in seconds.  Returns the number of updates written, or -1
 * if cap is too small or memory runs out.
 */
typedef struct {
    uint64_t *key;   /* ~0 empty, ~1 tombstone */
    int64_t *val;
    uint64_t mask;
} gg_map;

#define GG_EMPTY (~0ULL)
#define GG_TOMB (~1ULL)

static int map_init(gg_map *m, uint64_t items) {
    uint64_t cap = 16;
    while (cap < 4 * items + 16) cap <<= 1;
    m->key = (uint64_t *)malloc(cap * sizeof(uint64_t));
    m->val = (int64_t *)malloc(cap * sizeof(int64_t));
    if (!m->key || !m->val) return -1;
    memset(m->key, 0xff, cap * sizeof(uint64_t));
    m->mask = cap - 1;
    return 0;
}

static void map_free(gg_map *m) {
    free(m->key);
    free(m->val);
}

/* slot of key, or -1 */
static int64_t map_find(const gg_map *m, uint64_t key) {
    uint64_t h = mix64(key) & m->mask;
    while (m->key[h] != GG_EMPTY) {
        if (m->key[h] == key) return (int64_t)h;
        h = (h + 1) & m->mask;
    }
    return -1;
}

static void map_put(gg_map *m, uint64_t key, int64_t val) {
    int64_t s = map_find(m, key);
    if (s >= 0) {
        m->val[s] = val;
        return;
    }
    uint64_t h = mix64(key) & m->mask;
    while (m->key[h] != GG_EMPTY && m->key[h] != GG_TOMB) h = (h + 1) & m->mask;
    m->key[h] = key;
    m->val[h] = val;
}

static void map_del(gg_map *m, uint64_t key) {
    int64_t s = map_find(m, key);
    if (s >= 0) m->key[s] = GG_TOMB;
}

static inline uint64_t pair_key(uint64_t a, uint64_t b) {
    return a < b ? (a << 32) | b : (b << 32) | a;
}

/* size of batch j: log-uniform in [min_size, max_size] */
static int64_t stream_size(int64_t j, int64_t min_size, int64_t max_size, uint64_t seed) {
    const double lo = log((double)min_size), hi = log((double)max_size + 1.0);
    int64_t m = (int64_t)floor(exp(lo + (hi - lo) * unit(draw(seed, 21, (uint64_t)j))));
    if (m < min_size) m = min_size;
    if (m > max_size) m = max_size;
    return m;
}

/* total number of updates gg_stream draws (the capacity it needs) */
int64_t gg_stream_total(int64_t batches, int64_t min_size, int64_t max_size, uint64_t seed) {
    int64_t s = 0;
    for (int64_t j = 0; j < batches; ++j) s += stream_size(j, min_size, max_size, seed);
    return s;
}

int64_t gg_stream(int64_t n, const int64_t *rowptr, const int32_t *col, int64_t deg_bound, int64_t batches,
                  int64_t min_size, int64_t max_size, double p_insert, double rate, uint64_t seed,
                  int64_t cap, int64_t *offsets, int32_t *src, int32_t *dst, uint8_t *is_insert,
                  double *arrival) {
    const int64_t nnz = rowptr[n];
    int64_t *deg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint64_t *ins_list = (uint64_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(uint64_t));
    int32_t *bdeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));  /* inserts so far in the batch */
    gg_map deleted = {0}, inserted = {0}, in_batch = {0};
    int64_t n_ins = 0, out = 0, rc = 0;
    double t_arr = 0.0;
    uint64_t t = 0;
    if (!deg || !ins_list || !bdeg || map_init(&deleted, (uint64_t)cap) || map_init(&inserted, (uint64_t)cap) ||
        map_init(&in_batch, (uint64_t)(max_size > 0 ? max_size : 1))) {
        rc = -1;
        goto done;
    }
    for (int64_t v = 0; v < n; ++v) deg[v] = rowptr[v + 1] - rowptr[v];
    offsets[0] = 0;
    for (int64_t j = 0; j < batches; ++j) {
        /* arrival and size */
        t_arr += -log(1.0 - unit(draw(seed, 20, (uint64_t)j))) / rate;
        arrival[j] = t_arr;
        const int64_t m = stream_size(j, min_size, max_size, seed);
        if (out + m > cap) {
            rc = -1;
            goto done;
        }
        const int64_t b0 = out;
        int64_t guard = 0;
        while (out - b0 < m && guard < 1000 * (m + 10)) {
            ++guard;
            ++t;
            const int ins = unit(draw(seed, 22, t)) < p_insert;
            uint64_t a, b;
            if (ins) {
                a = below(draw(seed, 23, t), (uint64_t)n);
                b = below(draw(seed, 24, t), (uint64_t)n);
                if (a == b) continue;
                if (deg[a] + bdeg[a] >= deg_bound || deg[b] + bdeg[b] >= deg_bound) continue;
                const uint64_t key = pair_key(a, b);
                const int in_base = has_arc(rowptr, col, (int32_t)a, (int32_t)b);
                const int alive = (in_base && map_find(&deleted, key) < 0) || map_find(&inserted, key) >= 0;
                if (alive || map_find(&in_batch, key) >= 0) continue;
                map_put(&in_batch, key, 1);
                ++bdeg[a];
                ++bdeg[b];
            } else {
                const uint64_t slots = (uint64_t)nnz + 2 * (uint64_t)n_ins;
                if (slots == 0) continue;
                const uint64_t x = below(draw(seed, 25, t), slots);
                if (x < (uint64_t)nnz) {
                    int64_t l = 0, h = n;
                    while (h - l > 1) {
                        int64_t mid = (l + h) >> 1;
                        if ((uint64_t)rowptr[mid] <= x) l = mid; else h = mid;
                    }
                    a = (uint64_t)l;
                    b = (uint64_t)col[x];
                    if (map_find(&deleted, pair_key(a, b)) >= 0) continue;
                } else {
                    const uint64_t key = ins_list[(x - (uint64_t)nnz) / 2];
                    a = key >> 32;
                    b = key & 0xffffffffULL;
                }
                const uint64_t key = pair_key(a, b);
                if (map_find(&in_batch, key) >= 0) continue;
                map_put(&in_batch, key, 0);
            }
            src[out] = (int32_t)a;
            dst[out] = (int32_t)b;
            is_insert[out] = (uint8_t)ins;
            ++out;
        }
        /* apply the batch to the evolving edge set */
        memset(in_batch.key, 0xff, (in_batch.mask + 1) * sizeof(uint64_t));
        for (int64_t e = b0; e < out; ++e) {
            const uint64_t a = (uint64_t)src[e], b = (uint64_t)dst[e], key = pair_key(a, b);
            if (is_insert[e]) {
                bdeg[a] = 0;
                bdeg[b] = 0;
                ++deg[a];
                ++deg[b];
                if (map_find(&deleted, key) >= 0) {
                    map_del(&deleted, key);        /* a deleted base edge comes back */
                } else {
                    ins_list[n_ins] = key;
                    map_put(&inserted, key, n_ins);
                    ++n_ins;
                }
            } else {
                --deg[a];
                --deg[b];
                const int64_t s = map_find(&inserted, key);
                if (s >= 0) {                      /* swap-remove from the inserted list */
                    const int64_t slot = inserted.val[s];
                    map_del(&inserted, key);
                    --n_ins;
                    if (slot != n_ins) {
                        ins_list[slot] = ins_list[n_ins];
                        map_put(&inserted, ins_list[slot], slot);
                    }
                } else {
                    map_put(&deleted, key, 1);
                }
            }
        }
        offsets[j + 1] = out;
    }
    rc = out;
done:
    free(deg);
    free(ins_list);
    free(bdeg);
    if (deleted.key) map_free(&deleted);
    if (inserted.key) map_free(&inserted);
    if (in_batch.key) map_free(&in_batch);
    return rc;
}
