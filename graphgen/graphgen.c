/*
 * Seeded synthetic input generators: RMAT graphs (directed or symmetrised)
 * delivered as an in-edge CSR, and Netflix-shaped bipartite rating graphs.
 *
 * These produce the INPUTS shared by the FP64 oracle and by the CUDA path.
 * They contain none of the method's arithmetic (no PageRank, no segmenting,
 * no clustering): only random-number draws, edge generation, cleanup
 * (self-loops and duplicates dropped) and the CSR layout of the result.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014; constants as published by
 * Vigna).  A "stream (seed, i)" starts from state mix64(mix64(seed) + i) and
 * every draw adds the golden gamma and returns mix64 of the state.
 *
 * RMAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge descends `scale`
 * levels of the adjacency matrix; at each level one 64-bit draw u picks a
 * quadrant: u < A -> (0,0), u < A+B -> (0,1), u < A+B+C -> (1,0), else (1,1),
 * with the thresholds floor(p * 2^64) computed once in double precision.
 * The first bit is the source's, the second the destination's.  Edge i uses
 * stream (seed, i).  Vertex IDs are then permuted by a Fisher-Yates shuffle
 * drawn from stream (seed + 1, 0).
 *
 * Host code only; same results on x86-64 and aarch64 (no intrinsics; the
 * only floating point is in the bipartite generator's degree draws).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } sm64;

static inline sm64 stream_at(uint64_t seed, uint64_t i) {
    sm64 r; r.s = mix64(mix64(seed) + i); return r;
}
static inline uint64_t next64(sm64 *g) {
    g->s += GOLDEN_GAMMA;
    return mix64(g->s);
}
/* uniform integer in [0, n) by the multiply-high method (Lemire) */
static inline uint64_t below(sm64 *g, uint64_t n) {
    return (uint64_t)(((unsigned __int128)next64(g) * n) >> 64);
}
/* uniform double in [0,1) from the top 53 bits */
static inline double unit(sm64 *g) {
    return (double)(next64(g) >> 11) * (1.0 / 9007199254740992.0);
}

int gg_splitmix_draws(uint64_t seed, uint64_t i, int32_t n, uint64_t *out) {
    sm64 g = stream_at(seed, i);
    for (int32_t j = 0; j < n; ++j) out[j] = next64(&g);
    return 0;
}

/* Row v of an n x K matrix: K uniform draws in [0, hi) from stream (seed, v). */
int gg_uniform_rows(uint64_t seed, int64_t n, int32_t K, double hi, double *out) {
    if (n < 0 || K < 1) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        sm64 g = stream_at(seed, (uint64_t)v);
        for (int32_t k = 0; k < K; ++k) out[v * K + k] = unit(&g) * hi;
    }
    return 0;
}

/* Fisher-Yates shuffle of 0..n-1 from stream (seed, 0): perm[old] = new. */
int gg_permutation(uint64_t seed, int64_t n, int32_t *perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    sm64 g = stream_at(seed, 0);
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)below(&g, (uint64_t)i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_i32(int32_t *a, int64_t n) {
    if (n < 32) {
        for (int64_t i = 1; i < n; ++i) {
            int32_t x = a[i]; int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
            a[j + 1] = x;
        }
    } else {
        qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Build a cleaned in-edge CSR from an edge list (src[i] -> dst[i]):
 * rows are destinations, each row's sources sorted ascending, self-loops
 * and duplicates removed.  Returns E after cleanup; *out_src is malloc'ed
 * and owned by the caller (free with gg_free).
 */
static int64_t edges_to_in_csr(int64_t V, int64_t M, const int32_t *esrc,
                               const int32_t *edst, int64_t *offsets,
                               int32_t **out_src) {
    int64_t *cnt = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    if (!cnt) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i)
        __atomic_fetch_add(&cnt[edst[i] + 1], 1, __ATOMIC_RELAXED);
    for (int64_t v = 0; v < V; ++v) cnt[v + 1] += cnt[v];
    int32_t *tmp = (int32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    int64_t *cur = (int64_t *)malloc((size_t)(V + 1) * sizeof(int64_t));
    if (!tmp || !cur) { free(cnt); free(tmp); free(cur); return -1; }
    memcpy(cur, cnt, (size_t)(V + 1) * sizeof(int64_t));
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        int64_t p = __atomic_fetch_add(&cur[edst[i]], 1, __ATOMIC_RELAXED);
        tmp[p] = esrc[i];
    }
    /* sort + dedupe + drop self-loops per row; new lengths into cur[v] */
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < V; ++v) {
        int32_t *row = tmp + cnt[v];
        int64_t n = cnt[v + 1] - cnt[v];
        sort_i32(row, n);
        int64_t w = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (row[j] == (int32_t)v) continue;
            if (w > 0 && row[w - 1] == row[j]) continue;
            row[w++] = row[j];
        }
        cur[v] = w;
    }
    offsets[0] = 0;
    for (int64_t v = 0; v < V; ++v) offsets[v + 1] = offsets[v] + cur[v];
    int64_t E = offsets[V];
    int32_t *src = (int32_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(int32_t));
    if (!src) { free(cnt); free(tmp); free(cur); return -1; }
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < V; ++v)
        memcpy(src + offsets[v], tmp + cnt[v], (size_t)cur[v] * sizeof(int32_t));
    free(cnt); free(tmp); free(cur);
    *out_src = src;
    return E;
}

/*
 * RMAT graph of 2^scale vertices and edge_factor * 2^scale generated edges.
 * symmetric != 0 adds the reverse of every generated edge (undirected graph
 * stored as arcs in both directions).  permute != 0 relabels vertices by
 * gg_permutation(seed + 1).  offsets must hold 2^scale + 1 entries.
 * Returns E after cleanup (or -1 on allocation failure); *out_src receives
 * a malloc'ed int32[E] that the caller releases with gg_free.
 */
int64_t gg_rmat_in_csr(int32_t scale, int32_t edge_factor, double a, double b,
                       double c, uint64_t seed, int32_t symmetric,
                       int32_t permute, int64_t *offsets, int32_t **out_src) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    const int64_t V = (int64_t)1 << scale;
    const int64_t G = (int64_t)edge_factor * V;
    const int64_t M = symmetric ? 2 * G : G;
    const double two64 = 18446744073709551616.0;
    const uint64_t tA = (uint64_t)(a * two64);
    const uint64_t tAB = (uint64_t)((a + b) * two64);
    const uint64_t tABC = (uint64_t)((a + b + c) * two64);
    int32_t *perm = NULL;
    if (permute) {
        perm = (int32_t *)malloc((size_t)V * sizeof(int32_t));
        if (!perm) return -1;
        gg_permutation(seed + 1, V, perm);
    }
    int32_t *es = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    int32_t *ed = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    if (!es || !ed) { free(perm); free(es); free(ed); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < G; ++i) {
        sm64 g = stream_at(seed, (uint64_t)i);
        uint32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; ++l) {
            uint64_t r = next64(&g);
            uint32_t bu, bv;
            if (r < tA) { bu = 0; bv = 0; }
            else if (r < tAB) { bu = 0; bv = 1; }
            else if (r < tABC) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        int32_t su = perm ? perm[u] : (int32_t)u;
        int32_t sv = perm ? perm[v] : (int32_t)v;
        es[i] = su; ed[i] = sv;
        if (symmetric) { es[G + i] = sv; ed[G + i] = su; }
    }
    free(perm);
    int64_t E = edges_to_in_csr(V, M, es, ed, offsets, out_src);
    free(es); free(ed);
    return E;
}

/* Generic cleanup of a caller-supplied edge list into an in-edge CSR. */
int64_t gg_edges_in_csr(int64_t V, int64_t M, const int32_t *esrc,
                        const int32_t *edst, int64_t *offsets,
                        int32_t **out_src) {
    return edges_to_in_csr(V, M, esrc, edst, offsets, out_src);
}

/*
 * Netflix-shaped bipartite rating graph, stored user-major:
 * user_offsets[U+1], items[R] (ascending within a user), ratings[R] in 1..5.
 *  - user degrees: lognormal(mu, sigma) draws (Box-Muller on stream
 *    (seed, 0)), scaled so they total R_target, rounded by largest
 *    remainder, clipped to [1, I]; the clipping surplus/deficit is then
 *    settled one unit at a time over users in index order until the total
 *    is exactly R_target (when feasible);
 *  - items of user u: drawn from Zipf(s) over item ranks 0..I-1 without
 *    replacement from stream (seed + 2, u): rejection of repeats while the
 *    user's degree is at most I/4, otherwise Efraimidis-Spirakis keys over
 *    all items (exponential-clock form) keeping the d smallest;
 *  - item popularity rank r is mapped to item id by a permutation drawn
 *    from stream (seed + 3, 0);
 *  - rating: uniform in 1..5 from stream (seed + 4, u).
 * Returns R (total ratings) or -1.  Arrays are caller-allocated: offsets of
 * U+1, items and ratings of R_target entries.
 */
static int cmp_u64key(const void *a, const void *b) {
    const double *x = (const double *)a, *y = (const double *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

int64_t gg_bipartite(int64_t U, int64_t I, int64_t R_target, double mu,
                     double sigma, double zipf_s, uint64_t seed,
                     int64_t *user_offsets, int32_t *items, uint8_t *ratings) {
    if (U < 1 || I < 1 || R_target < U || R_target > U * I) return -1;
    double *w = (double *)malloc((size_t)U * sizeof(double));
    int64_t *deg = (int64_t *)malloc((size_t)U * sizeof(int64_t));
    double *cdf = (double *)malloc((size_t)I * sizeof(double));
    int32_t *ipm = (int32_t *)malloc((size_t)I * sizeof(int32_t));
    if (!w || !deg || !cdf || !ipm) { free(w); free(deg); free(cdf); free(ipm); return -1; }
    sm64 g = stream_at(seed, 0);
    double tot = 0.0;
    for (int64_t u = 0; u < U; u += 2) {
        double u1 = unit(&g), u2 = unit(&g);
        if (u1 < 1e-300) u1 = 1e-300;
        double rad = sqrt(-2.0 * log(u1));
        double z0 = rad * cos(6.283185307179586 * u2);
        double z1 = rad * sin(6.283185307179586 * u2);
        w[u] = exp(mu + sigma * z0); tot += w[u];
        if (u + 1 < U) { w[u + 1] = exp(mu + sigma * z1); tot += w[u + 1]; }
    }
    /* largest remainder rounding to R_target */
    double scale = (double)R_target / tot;
    int64_t assigned = 0;
    for (int64_t u = 0; u < U; ++u) {
        double x = w[u] * scale;
        deg[u] = (int64_t)floor(x);
        w[u] = x - (double)deg[u];
        assigned += deg[u];
    }
    {
        int64_t left = R_target - assigned;
        /* give one unit to the `left` users with the largest remainders
           (ties by lower index): selection by repeated passes over a sorted
           index is avoided with a threshold search on the remainder. */
        if (left > 0) {
            double lo = 0.0, hi = 1.0;
            for (int it = 0; it < 64; ++it) {
                double mid = 0.5 * (lo + hi);
                int64_t n = 0;
                for (int64_t u = 0; u < U; ++u) n += (w[u] > mid);
                if (n > left) lo = mid; else hi = mid;
            }
            for (int64_t u = 0; u < U && left > 0; ++u)
                if (w[u] > hi) { deg[u]++; left--; }
            for (int64_t u = 0; u < U && left > 0; ++u)
                if (w[u] <= hi && w[u] > lo) { deg[u]++; left--; }
            for (int64_t u = 0; u < U && left > 0; ++u)
                if (w[u] <= lo) { deg[u]++; left--; }
        }
    }
    /* clip to [1, I] and settle the total exactly */
    int64_t total = 0;
    for (int64_t u = 0; u < U; ++u) {
        if (deg[u] < 1) deg[u] = 1;
        if (deg[u] > I) deg[u] = I;
        total += deg[u];
    }
    for (int pass = 0; total != R_target && pass < 1000000; ++pass) {
        int changed = 0;
        for (int64_t u = 0; u < U && total != R_target; ++u) {
            if (total < R_target && deg[u] < I && deg[u] > 1) { deg[u]++; total++; changed = 1; }
            else if (total > R_target && deg[u] > 1) { deg[u]--; total--; changed = 1; }
        }
        if (!changed) break;
    }
    user_offsets[0] = 0;
    for (int64_t u = 0; u < U; ++u) user_offsets[u + 1] = user_offsets[u] + deg[u];
    int64_t R = user_offsets[U];
    /* Zipf CDF over ranks */
    double acc = 0.0;
    for (int64_t r = 0; r < I; ++r) { acc += pow((double)(r + 1), -zipf_s); cdf[r] = acc; }
    for (int64_t r = 0; r < I; ++r) cdf[r] /= acc;
    gg_permutation(seed + 3, I, ipm);
    #pragma omp parallel
    {
        double *keys = (double *)malloc((size_t)I * 2 * sizeof(double));
        uint8_t *seen = (uint8_t *)calloc((size_t)I, 1);
        int64_t *ranks = (int64_t *)malloc((size_t)I * sizeof(int64_t));
        #pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < U; ++u) {
            int64_t d = deg[u];
            int32_t *out = items + user_offsets[u];
            sm64 gu = stream_at(seed + 2, (uint64_t)u);
            if (d * 4 <= I) {
                int64_t n = 0;
                while (n < d) {
                    double x = unit(&gu);
                    int64_t lo2 = 0, hi2 = I - 1;
                    while (lo2 < hi2) { int64_t m = (lo2 + hi2) / 2; if (cdf[m] > x) hi2 = m; else lo2 = m + 1; }
                    if (!seen[lo2]) { seen[lo2] = 1; ranks[n] = lo2; out[n++] = ipm[lo2]; }
                }
                for (int64_t j = 0; j < d; ++j) seen[ranks[j]] = 0;
            } else {
                for (int64_t r = 0; r < I; ++r) {
                    double p = cdf[r] - (r ? cdf[r - 1] : 0.0);
                    double e = -log(1.0 - unit(&gu));
                    keys[2 * r] = e / p;
                    keys[2 * r + 1] = (double)r;
                }
                qsort(keys, (size_t)I, 2 * sizeof(double), cmp_u64key);
                for (int64_t j = 0; j < d; ++j) out[j] = ipm[(int64_t)keys[2 * j + 1]];
            }
            sort_i32(out, d);
            sm64 gr = stream_at(seed + 4, (uint64_t)u);
            for (int64_t j = 0; j < d; ++j) ratings[user_offsets[u] + j] = (uint8_t)(1 + below(&gr, 5));
        }
        free(keys); free(seen); free(ranks);
    }
    free(w); free(deg); free(cdf); free(ipm);
    return R;
}

void gg_free(void *p) { free(p); }

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
