/*
 * gen.c -- seeded synthetic inputs: graphs (R-MAT, Barabasi-Albert, Erdos-Renyi) in
 * in-CSR form (row = target node, columns = source nodes, sorted ascending within a
 * row) and uniformly random seed-node sets.
 *
 * This module holds none of the propagation method's arithmetic.  Its randomness is
 * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) applied to a counter, so every output is a pure function of (seed,
 * index) and does not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static inline uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* stream-separated counter hash */
static inline uint64_t hash3(uint64_t seed, uint64_t stream, uint64_t i)
{
    return mix64(mix64(seed ^ (stream * 0xD6E8FEB86659FD93ull)) + i);
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------ R-MAT */

typedef struct {
    int scale;
    uint64_t n_edges;
    uint64_t tA, tAB, tABC; /* cumulative quadrant thresholds scaled to 2^32 */
    uint64_t seed;
    int32_t *row_ptr;       /* [n+1] */
    int32_t *col_idx;       /* [E] */
    uint32_t *cursor;       /* [n] scatter cursor / degree counter */
    int nthreads;
    int phase;
} rmat_job;

typedef struct { rmat_job *job; int tid; } rmat_worker;

static inline void rmat_edge(const rmat_job *jb, uint64_t i, uint32_t *src, uint32_t *dst)
{
    uint32_t s = 0, d = 0;
    uint64_t h = 0;
    for (int lvl = 0; lvl < jb->scale; ++lvl) {
        if ((lvl & 1) == 0) h = hash3(jb->seed, 1 + (uint64_t)(lvl >> 1), i);
        uint64_t r = (lvl & 1) ? (h >> 32) : (h & 0xFFFFFFFFull);
        uint32_t sb, db;
        if (r < jb->tA) { sb = 0; db = 0; }
        else if (r < jb->tAB) { sb = 0; db = 1; }
        else if (r < jb->tABC) { sb = 1; db = 0; }
        else { sb = 1; db = 1; }
        s = (s << 1) | sb;
        d = (d << 1) | db;
    }
    *src = s;
    *dst = d;
}

static void *rmat_worker_main(void *arg)
{
    rmat_worker *w = (rmat_worker *)arg;
    rmat_job *jb = w->job;
    const uint64_t n = 1ull << jb->scale;
    uint64_t lo = jb->n_edges * (uint64_t)w->tid / (uint64_t)jb->nthreads;
    uint64_t hi = jb->n_edges * (uint64_t)(w->tid + 1) / (uint64_t)jb->nthreads;
    if (jb->phase == 0) {          /* count in-degrees */
        for (uint64_t i = lo; i < hi; ++i) {
            uint32_t s, d;
            rmat_edge(jb, i, &s, &d);
            __atomic_fetch_add(&jb->cursor[d], 1u, __ATOMIC_RELAXED);
        }
    } else if (jb->phase == 1) {   /* scatter sources */
        for (uint64_t i = lo; i < hi; ++i) {
            uint32_t s, d;
            rmat_edge(jb, i, &s, &d);
            uint32_t pos = __atomic_fetch_add(&jb->cursor[d], 1u, __ATOMIC_RELAXED);
            jb->col_idx[(uint64_t)jb->row_ptr[d] + pos] = (int32_t)s;
        }
    } else {                       /* sort each row: the order becomes deterministic */
        uint64_t vlo = n * (uint64_t)w->tid / (uint64_t)jb->nthreads;
        uint64_t vhi = n * (uint64_t)(w->tid + 1) / (uint64_t)jb->nthreads;
        for (uint64_t v = vlo; v < vhi; ++v) {
            int32_t b = jb->row_ptr[v], e = jb->row_ptr[v + 1];
            if (e - b > 1) qsort(jb->col_idx + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        }
    }
    return NULL;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): 2^scale nodes, n_edges arcs, each
 * arc picks one quadrant per level with probabilities (a, b, c, 1-a-b-c); b is the
 * (src bit 0, dst bit 1) quadrant.  Duplicates and self-loops are kept.  row_ptr must
 * hold 2^scale+1 entries and col_idx n_edges entries (n_edges < 2^31). */
int gen_rmat(int scale, uint64_t n_edges, double a, double b, double c, uint64_t seed,
             int nthreads, int32_t *row_ptr, int32_t *col_idx)
{
    if (scale < 1 || scale > 30 || n_edges >= (1ull << 31) || nthreads < 1) return -1;
    const uint64_t n = 1ull << scale;
    rmat_job jb;
    memset(&jb, 0, sizeof jb);
    jb.scale = scale;
    jb.n_edges = n_edges;
    jb.tA = (uint64_t)(a * 4294967296.0);
    jb.tAB = (uint64_t)((a + b) * 4294967296.0);
    jb.tABC = (uint64_t)((a + b + c) * 4294967296.0);
    jb.seed = seed;
    jb.row_ptr = row_ptr;
    jb.col_idx = col_idx;
    jb.nthreads = nthreads;
    jb.cursor = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!jb.cursor) return -2;
    rmat_worker *ws = (rmat_worker *)calloc((size_t)nthreads, sizeof(rmat_worker));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int phase = 0; phase < 3; ++phase) {
        jb.phase = phase;
        if (phase == 1) {
            row_ptr[0] = 0;
            for (uint64_t v = 0; v < n; ++v) row_ptr[v + 1] = row_ptr[v] + (int32_t)jb.cursor[v];
            memset(jb.cursor, 0, n * sizeof(uint32_t));
        }
        for (int i = 0; i < nthreads; ++i) {
            ws[i].job = &jb;
            ws[i].tid = i;
            pthread_create(&th[i], NULL, rmat_worker_main, &ws[i]);
        }
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    }
    free(ws);
    free(th);
    free(jb.cursor);
    return 0;
}

/* --------------------------------------------------- undirected edge lists */

/* Build an in-CSR from arcs (src[i] -> dst[i]); columns sorted within each row. */
static int build_in_csr(int32_t n, int64_t n_arcs, const int32_t *src, const int32_t *dst,
                        int32_t *row_ptr, int32_t *col_idx)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -2;
    for (int64_t i = 0; i < n_arcs; ++i) cnt[dst[i] + 1]++;
    for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    for (int32_t v = 0; v <= n; ++v) row_ptr[v] = (int32_t)cnt[v];
    for (int64_t i = 0; i < n_arcs; ++i) col_idx[cnt[dst[i]]++] = src[i];
    for (int32_t v = 0; v < n; ++v) {
        int32_t b = row_ptr[v], e = row_ptr[v + 1];
        if (e - b > 1) qsort(col_idx + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
    }
    free(cnt);
    return 0;
}

/* Barabasi-Albert (preferential attachment): nodes 0..m form a clique; every later
 * node v attaches to m distinct earlier nodes, each drawn with probability
 * proportional to its current degree (uniform pick from the list of edge endpoints).
 * Both arc directions are stored, so in-degree = degree.  Arc count = 2*(m(m+1)/2 +
 * (n-m-1)*m); row_ptr has n+1 entries, col_idx that many arcs. */
int64_t gen_ba_arcs(int32_t n, int32_t m)
{
    if (m < 1 || n < m + 1) return -1;
    return 2 * ((int64_t)m * (m + 1) / 2 + (int64_t)(n - m - 1) * m);
}

int gen_ba(int32_t n, int32_t m, uint64_t seed, int32_t *row_ptr, int32_t *col_idx)
{
    int64_t n_arcs = gen_ba_arcs(n, m);
    if (n_arcs < 0) return -1;
    int64_t n_und = n_arcs / 2;
    int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n_und));
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_arcs);
    int32_t *dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_arcs);
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    if (!ends || !src || !dst || !pick) { free(ends); free(src); free(dst); free(pick); return -2; }
    int64_t ne = 0, na = 0;
    for (int32_t i = 0; i <= m; ++i)
        for (int32_t j = i + 1; j <= m; ++j) {
            ends[ne++] = i; ends[ne++] = j;
            src[na] = i; dst[na++] = j;
            src[na] = j; dst[na++] = i;
        }
    uint64_t draw = 0;
    for (int32_t v = m + 1; v < n; ++v) {
        int got = 0;
        while (got < m) {
            uint64_t h = hash3(seed, 7, draw++);
            int32_t t = ends[h % (uint64_t)ne];
            int dup = 0;
            for (int q = 0; q < got; ++q) if (pick[q] == t) { dup = 1; break; }
            if (!dup) pick[got++] = t;
        }
        for (int q = 0; q < m; ++q) {
            ends[ne++] = v; ends[ne++] = pick[q];
            src[na] = v; dst[na++] = pick[q];
            src[na] = pick[q]; dst[na++] = v;
        }
    }
    int rc = build_in_csr(n, na, src, dst, row_ptr, col_idx);
    free(ends); free(src); free(dst); free(pick);
    return rc;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Erdos-Renyi, undirected, simple.  n <= 100000: G(n, p) with p = mean_deg/(n-1),
 * every pair {i<j} kept iff its hash falls below p*2^64.  Larger n: G(n, M) with
 * M = round(mean_deg*n/2) distinct pairs drawn by hashing.  Both arc directions are
 * stored.  Returns the arc count through *n_arcs_out; pass row_ptr/col_idx = NULL to
 * query the size first (the same seed gives the same graph on the second call). */
int gen_er(int32_t n, double mean_deg, uint64_t seed, int64_t *n_arcs_out,
           int32_t *row_ptr, int32_t *col_idx)
{
    if (n < 2 || mean_deg < 0) return -1;
    uint64_t *pairs = NULL;
    int64_t np = 0, cap = 0;
    if (n <= 100000) {
        double p = mean_deg / (double)(n - 1);
        uint64_t thr = p >= 1.0 ? UINT64_MAX : (uint64_t)(p * 18446744073709551616.0);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j) {
                if (hash3(seed, 11, (uint64_t)i * (uint64_t)n + (uint64_t)j) < thr) {
                    if (np == cap) {
                        cap = cap ? 2 * cap : 1024;
                        pairs = (uint64_t *)realloc(pairs, sizeof(uint64_t) * (size_t)cap);
                        if (!pairs) return -2;
                    }
                    pairs[np++] = ((uint64_t)i << 32) | (uint64_t)j;
                }
            }
    } else {
        int64_t M = (int64_t)(mean_deg * (double)n / 2.0 + 0.5);
        cap = M + 16;
        pairs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)cap);
        if (!pairs) return -2;
        uint64_t draw = 0;
        while (np < M) {
            int64_t want = M - np;
            for (int64_t q = 0; q < want; ++q) {
                uint64_t h = hash3(seed, 13, draw++);
                uint32_t u = (uint32_t)((h & 0xFFFFFFFFull) % (uint64_t)n);
                uint32_t v = (uint32_t)((h >> 32) % (uint64_t)n);
                if (u == v) continue;
                if (u > v) { uint32_t t = u; u = v; v = t; }
                pairs[np++] = ((uint64_t)u << 32) | v;
            }
            qsort(pairs, (size_t)np, sizeof(uint64_t), cmp_u64);
            int64_t k = 0;
            for (int64_t q = 0; q < np; ++q)
                if (q == 0 || pairs[q] != pairs[q - 1]) pairs[k++] = pairs[q];
            np = k;
        }
        /* keep exactly M: drop the largest surplus (there is none: we top up to M) */
    }
    int64_t n_arcs = 2 * np;
    *n_arcs_out = n_arcs;
    if (!row_ptr || !col_idx) { free(pairs); return 0; }
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_arcs ? n_arcs : 1));
    int32_t *dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_arcs ? n_arcs : 1));
    if (!src || !dst) { free(pairs); free(src); free(dst); return -2; }
    for (int64_t q = 0; q < np; ++q) {
        int32_t u = (int32_t)(pairs[q] >> 32), v = (int32_t)(pairs[q] & 0xFFFFFFFFull);
        src[2 * q] = u; dst[2 * q] = v;
        src[2 * q + 1] = v; dst[2 * q + 1] = u;
    }
    int rc = build_in_csr(n, n_arcs, src, dst, row_ptr, col_idx);
    free(pairs); free(src); free(dst);
    return rc;
}

/* k distinct nodes drawn uniformly from 0..n-1 (partial Fisher-Yates), sorted. */
int gen_seed_set(int32_t n, int32_t k, uint64_t seed, int32_t *out)
{
    if (k < 0 || k > n) return -1;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!perm) return -2;
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = 0; i < k; ++i) {
        uint64_t h = hash3(seed, 17, (uint64_t)i);
        int32_t j = i + (int32_t)(h % (uint64_t)(n - i));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        out[i] = perm[i];
    }
    qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
    free(perm);
    return 0;
}

/* Raw counter hash, exposed so that harness code can draw reproducible parameters. */
uint64_t gen_hash(uint64_t seed, uint64_t stream, uint64_t i)
{
    return hash3(seed, stream, i);
}
