/*
 * FP64 CPU ORACLE for the segmented pull gather of "Making Caches Work for
 * Graph Analytics" (Cagra).  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the product path
 * never does.  Plain, slow, sequential-order loops written from the paper's
 * definitions; it shares no code with the CUDA library.  OpenMP only splits
 * independent destination rows, so every per-row sum keeps its left-to-right
 * CSR order and results do not depend on the thread count.
 *
 * Graph convention: in-edge CSR.  Row v of (offsets, src) lists the sources
 * u of the edges u -> v, in CSR order (Section II-A: vertexArray / edgeArray).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Out-degree of every vertex = number of CSR entries naming it as source
 * (the `degree` array of Algorithm 1). */
void orc_out_degree(int64_t V, const int64_t *offsets, const int32_t *src,
                    int64_t *outdeg) {
    for (int64_t u = 0; u < V; ++u) outdeg[u] = 0;
    for (int64_t e = 0; e < offsets[V]; ++e) outdeg[src[e]]++;
}

/* Wall-clock seconds (OpenMP's timer when available). */
static double orc_now(void) {
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return (double)clock() / (double)CLOCKS_PER_SEC;
#endif
}

/*
 * One iteration of the plain pull update (Algorithm 1's gather with the
 * per-vertex update of Algorithm 5), from `rank` into `next`:
 *   D      = sum over u with outdeg(u) = 0 of rank[u]          (index order)
 *   c[u]   = rank[u] / outdeg(u)   (0 for a dangling u)
 *   S_v    = sum_{u -> v} c[u]                                 (CSR order)
 * seed < 0 (uniform teleport, dangling mass spread over all V vertices):
 *   next[v] = (1-d)/V + d (S_v + D/V)
 * seed >= 0 (personalised: teleport and dangling mass return to the seed):
 *   next[v] = d S_v,  then next[seed] += (1-d) + d D
 * `contrib` receives c.  Returns D.
 */
static double pr_step(int64_t V, const int64_t *offsets, const int32_t *src,
                      const int64_t *outdeg, double d, int64_t seed,
                      const double *rank, double *contrib, double *next) {
    const double base = (1.0 - d) / (double)V;
    double D = 0.0;
    for (int64_t u = 0; u < V; ++u)
        if (outdeg[u] == 0) D += rank[u];
    #pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < V; ++u)
        contrib[u] = outdeg[u] ? rank[u] / (double)outdeg[u] : 0.0;
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < V; ++v) {
        double s = 0.0;
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) s += contrib[src[e]];
        next[v] = seed < 0 ? base + d * (s + D / (double)V) : d * s;
    }
    if (seed >= 0) next[seed] += (1.0 - d) + d * D;
    return D;
}

/*
 * Plain pull PageRank (Algorithm 1's gather, with the per-vertex update of
 * Algorithm 5 in normalised form and uniform redistribution of the rank held
 * by dangling vertices):
 *   r_0 = 1/V
 *   D   = sum over u with outdeg(u) = 0 of r[u]            (index order)
 *   r'[v] = (1-d)/V + d * ( sum_{u -> v} r[u]/outdeg(u) + D/V )
 * `rank` holds the initial vector on entry (the caller fills 1/V for r_0)
 * and the result after `iters` iterations on exit.
 * resid[t] = sum_v |r_{t+1}[v] - r_t[v]| (index order); may be NULL.
 * iter_seconds[t] (may be NULL) = wall time of iteration t alone: the
 * out-degree pass and the allocations before the loop are not in it.
 */
int orc_pagerank(int64_t V, const int64_t *offsets, const int32_t *src,
                 int32_t iters, double d, double *rank, double *resid,
                 double *iter_seconds) {
    int64_t *outdeg = (int64_t *)malloc((size_t)V * sizeof(int64_t));
    double *contrib = (double *)malloc((size_t)V * sizeof(double));
    double *next = (double *)malloc((size_t)V * sizeof(double));
    if (!outdeg || !contrib || !next) { free(outdeg); free(contrib); free(next); return -1; }
    orc_out_degree(V, offsets, src, outdeg);
    for (int32_t t = 0; t < iters; ++t) {
        const double t0 = orc_now();
        pr_step(V, offsets, src, outdeg, d, -1, rank, contrib, next);
        double r = 0.0;
        for (int64_t v = 0; v < V; ++v) r += fabs(next[v] - rank[v]);
        if (resid) resid[t] = r;
        memcpy(rank, next, (size_t)V * sizeof(double));
        if (iter_seconds) iter_seconds[t] = orc_now() - t0;
    }
    free(outdeg); free(contrib); free(next);
    return 0;
}

/* gamma_m = m u / (1 - m u): the relative error bound of m roundings
 * (Higham, Accuracy and Stability of Numerical Algorithms, Lemma 3.1). */
static double orc_gamma(double m, double u) {
    return m > 0.0 ? m * u / (1.0 - m * u) : 0.0;
}

/*
 * The same iteration as orc_pagerank (seed < 0) or as one column of orc_ppr
 * (seed >= 0), started from r_0 = 1/V or from the one-hot seed vector, and
 * beside it a per-vertex bound on how far ANY evaluation of that iteration in
 * a binary floating-point format can drift from these FP64 values:
 *   u_acc    unit roundoff of the arithmetic (2^-24 for FP32): each product,
 *            each sum of two values and each conversion rounds once;
 *   u_store  relative rounding of the stored contributions c[u] beyond that
 *            (0 when they are kept in the arithmetic format; 2^-16 for a
 *            BF16 hi + lo pair, 2^-8 for BF16 alone).
 * The sum S_v of n = indeg(v) contributions may be associated in any order,
 * split across segments and merged: every such evaluation performs n - 1
 * additions of disjoint partial sums, so its rounding error is at most
 * gamma_{n-1} * (sum of the summands' magnitudes) (Higham, eq. 4.4 for any
 * summation tree).  With e_t[v] the bound after t iterations, the error of
 * the computed contributions is at most e_t[u]/outdeg(u) plus (2 u_acc +
 * u_store) c[u] (the reciprocal degree and the product round once each), the
 * dangling sum is off by at most the sum of e_t over dangling vertices plus
 * gamma_m D (the evaluation may form it from partial sums of up to m = 256
 * ranks in the arithmetic format before adding those in FP64), and the
 * update adds at most u_acc (4 d (S_v + Dsh_v) + r_{t+1}[v] + 7 Tsh_v),
 * where Dsh_v = D/V (uniform) or [v = seed] D is v's share of the dangling
 * mass and Tsh_v = (1-d)/V or [v = seed](1-d) its share of the teleport:
 * the conversion of the dangling share, the sum with S_v, the product with
 * d and the rounding of d itself (one u d (S_v + Dsh_v) each), the final sum
 * (u r_{t+1}), and the teleport constant, which is off by at most 7 u Tsh_v
 * even when (1-d)/V is formed in the arithmetic format from the rounded d
 * (d/(1-d) = 5.67 times d's rounding, plus the division).  Hence, to first
 * order,
 *   e_{t+1}[v] = (1 + g + 4u)(1 + 2u + u_store) * P_v + (1 + g + 8u) * rho_v
 *   P_v   = d sum_{u -> v} e_t[u]/outdeg(u) + d * (seed < 0 ? Ed/V : [v = seed] Ed)
 *   rho_v = (g + 2u + u_store) d S_v + u (4 d (S_v + Dsh_v) + r_{t+1}[v] + 7 Tsh_v)
 *           + gamma_m d Dsh_v + (gamma64_{n+8} + 2 gamma64_V) r_{t+1}[v]
 * with g = gamma_{n-1}(u_acc), Ed = sum of e_t over dangling vertices, and
 * the gamma64 terms covering this FP64 evaluation's own rounding (and the
 * FP64 dangling sums on both sides).  e_0 = u_acc r_0 (1/V rounded once; the
 * one-hot start is exact).  The factors (1 + ...) absorb the second-order
 * products of errors; a final factor 1 + 1e-9 covers using FP64 values for
 * the exact ones.  On exit rank holds r_iters and bound holds e_iters, so
 * |r_computed[v] - rank[v]| <= bound[v] for every vertex.
 * resid[t] (may be NULL) = sum_v |r_{t+1}[v] - r_t[v]| as in orc_pagerank.
 * iter_seconds[t] (may be NULL) = wall time of the plain iteration t alone
 * (pr_step and the copy; the bound's own work is not in it).
 */
int orc_pagerank_bound(int64_t V, const int64_t *offsets, const int32_t *src,
                       int32_t iters, double d, int64_t seed, double u_acc,
                       double u_store, double *rank, double *bound, double *resid,
                       double *iter_seconds) {
    if (V < 1 || seed >= V) return -2;
    const double u64 = ldexp(1.0, -53);
    const double gm = orc_gamma(256.0, u_acc);  /* FP32 partials of the dangling mass */
    int64_t *outdeg = (int64_t *)malloc((size_t)V * sizeof(int64_t));
    double *contrib = (double *)malloc((size_t)V * sizeof(double));
    double *next = (double *)malloc((size_t)V * sizeof(double));
    double *ce = (double *)malloc((size_t)V * sizeof(double));
    double *enext = (double *)malloc((size_t)V * sizeof(double));
    if (!outdeg || !contrib || !next || !ce || !enext) {
        free(outdeg); free(contrib); free(next); free(ce); free(enext);
        return -1;
    }
    orc_out_degree(V, offsets, src, outdeg);
    const double gV = 2.0 * orc_gamma((double)V, u64);
    for (int64_t v = 0; v < V; ++v) {
        rank[v] = seed < 0 ? 1.0 / (double)V : (v == seed ? 1.0 : 0.0);
        bound[v] = seed < 0 ? u_acc * rank[v] : 0.0;
    }
    for (int32_t t = 0; t < iters; ++t) {
        const double t0 = orc_now();
        const double Dm = pr_step(V, offsets, src, outdeg, d, seed, rank, contrib, next);
        if (iter_seconds) iter_seconds[t] = orc_now() - t0;
        double Ed = 0.0;
        for (int64_t u = 0; u < V; ++u)
            if (outdeg[u] == 0) Ed += bound[u];
        #pragma omp parallel for schedule(static)
        for (int64_t u = 0; u < V; ++u)
            ce[u] = outdeg[u] ? bound[u] / (double)outdeg[u] : 0.0;
        #pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t v = 0; v < V; ++v) {
            double S = 0.0, P = 0.0;
            for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
                S += contrib[src[e]];
                P += ce[src[e]];
            }
            const double n = (double)(offsets[v + 1] - offsets[v]);
            const double g = orc_gamma(n - 1.0, u_acc);
            P = d * P + (seed < 0 ? d * Ed / (double)V : (v == seed ? d * Ed : 0.0));
            const double Dsh = seed < 0 ? Dm / (double)V : (v == seed ? Dm : 0.0);
            const double Tsh = seed < 0 ? (1.0 - d) / (double)V : (v == seed ? 1.0 - d : 0.0);
            const double rho = (g + 2.0 * u_acc + u_store) * d * S +
                               u_acc * (4.0 * d * (S + Dsh) + next[v] + 7.0 * Tsh) +
                               gm * d * Dsh + (orc_gamma(n + 8.0, u64) + gV) * next[v];
            enext[v] = ((1.0 + g + 4.0 * u_acc) * (1.0 + 2.0 * u_acc + u_store) * P +
                        (1.0 + g + 8.0 * u_acc) * rho) * (1.0 + 1e-9);
        }
        if (resid) {
            double r = 0.0;
            for (int64_t v = 0; v < V; ++v) r += fabs(next[v] - rank[v]);
            resid[t] = r;
        }
        memcpy(rank, next, (size_t)V * sizeof(double));
        memcpy(bound, enext, (size_t)V * sizeof(double));
    }
    free(outdeg); free(contrib); free(next); free(ce); free(enext);
    return 0;
}

/*
 * Segment construction (Algorithm 2, Section III-A).  Source vertex u belongs
 * to segment s when bounds[s] <= u < bounds[s+1] (uniform bounds s*N give
 * Algorithm 2's segmentID = src / N).  For each segment, the subgraph keeps
 * every in-edge whose source lies in the segment, grouped by destination in
 * the parent CSR's row order (so already sorted by destination), with the
 * parent's edge order inside a row.
 *
 * Flat layout of all subgraphs, segment after segment:
 *   row_base[s]   first subgraph row of segment s (row_base[k] = total rows qV)
 *   edge_base[s]  first edge of segment s          (edge_base[k] = E)
 *   row_ptr[i]    first edge of subgraph row i      (row_ptr[qV] = E)
 *   col[e]        global source ID of edge e
 *   idx_map[i]    global destination ID of subgraph row i (idxMap)
 *   block_start[s*(nb+1) + b]  first local row (row - row_base[s]) of segment
 *                 s whose destination is >= b*B, for b = 0..nb (nb = ceil(V/B));
 *                 blockEnds[b] of Algorithm 4 is block_start[..b+1].
 * orc_segments_count fills row_base and edge_base; the caller then sizes the
 * arrays for orc_segments_fill.
 */
static int32_t *segment_of(int64_t V, int32_t k, const int64_t *bounds) {
    int32_t *seg = (int32_t *)malloc((size_t)(V > 0 ? V : 1) * sizeof(int32_t));
    if (!seg) return NULL;
    for (int32_t s = 0; s < k; ++s)
        for (int64_t u = bounds[s]; u < bounds[s + 1]; ++u) seg[u] = s;
    return seg;
}

int orc_segments_count(int64_t V, const int64_t *offsets, const int32_t *src,
                       int32_t k, const int64_t *bounds, int64_t *row_base,
                       int64_t *edge_base) {
    int32_t *seg = segment_of(V, k, bounds);
    int64_t *rows = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int64_t *edges = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int64_t *last = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    if (!seg || !rows || !edges || !last) { free(seg); free(rows); free(edges); free(last); return -1; }
    for (int32_t s = 0; s < k; ++s) last[s] = -1;
    for (int64_t v = 0; v < V; ++v)
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            int32_t s = seg[src[e]];
            edges[s]++;
            if (last[s] != v) { last[s] = v; rows[s]++; }
        }
    row_base[0] = 0; edge_base[0] = 0;
    for (int32_t s = 0; s < k; ++s) {
        row_base[s + 1] = row_base[s] + rows[s];
        edge_base[s + 1] = edge_base[s] + edges[s];
    }
    free(seg); free(rows); free(edges); free(last);
    return 0;
}

int orc_segments_fill(int64_t V, const int64_t *offsets, const int32_t *src,
                      int32_t k, const int64_t *bounds, int64_t B,
                      const int64_t *row_base, const int64_t *edge_base,
                      int64_t *row_ptr, int32_t *col, int32_t *idx_map,
                      int32_t *block_start) {
    int32_t *seg = segment_of(V, k, bounds);
    int64_t *rnext = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    int64_t *enext = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    int64_t *last = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    if (!seg || !rnext || !enext || !last) { free(seg); free(rnext); free(enext); free(last); return -1; }
    for (int32_t s = 0; s < k; ++s) { rnext[s] = row_base[s]; enext[s] = edge_base[s]; last[s] = -1; }
    /* addInEdge(v, src) in parent order */
    for (int64_t v = 0; v < V; ++v)
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            int32_t s = seg[src[e]];
            if (last[s] != v) {
                last[s] = v;
                idx_map[rnext[s]] = (int32_t)v;
                row_ptr[rnext[s]] = enext[s];
                rnext[s]++;
            }
            col[enext[s]++] = src[e];
        }
    row_ptr[row_base[k]] = edge_base[k];
    /* block indices: first local row whose destination reaches b*B */
    const int64_t nb = (V + B - 1) / B;
    for (int32_t s = 0; s < k; ++s) {
        int64_t R = row_base[s + 1] - row_base[s];
        int64_t i = 0;
        for (int64_t b = 0; b <= nb; ++b) {
            int64_t lo = b * B;
            while (i < R && idx_map[row_base[s] + i] < lo) ++i;
            block_start[(int64_t)s * (nb + 1) + b] = (int32_t)(b == nb ? R : i);
        }
    }
    free(seg); free(rnext); free(enext); free(last);
    return 0;
}

/*
 * Segmented PageRank in FP64, in the paper's order: each iteration runs
 * parallel segment processing (Algorithm 3: subgraph after subgraph, each
 * row's partial sum over its edges left to right into intermBuf) and then the
 * cache-aware merge (Algorithm 4: per block of B destinations, output = 0,
 * then subgraph after subgraph add intermBuf[i] into output[idxMap[i]]),
 * then the same vertex update as orc_pagerank.
 */
int orc_pagerank_segmented(int64_t V, int32_t k, int64_t B,
                           const int64_t *row_base, const int64_t *row_ptr,
                           const int32_t *col, const int32_t *idx_map,
                           const int32_t *block_start, const int64_t *outdeg,
                           int32_t iters, double d, double *rank, double *resid) {
    const int64_t rows = row_base[k];
    const int64_t nb = (V + B - 1) / B;
    double *contrib = (double *)malloc((size_t)(V > 0 ? V : 1) * sizeof(double));
    double *interm = (double *)malloc((size_t)(rows > 0 ? rows : 1) * sizeof(double));
    double *out = (double *)malloc((size_t)(V > 0 ? V : 1) * sizeof(double));
    if (!contrib || !interm || !out) { free(contrib); free(interm); free(out); return -1; }
    const double base = (1.0 - d) / (double)V;
    for (int32_t t = 0; t < iters; ++t) {
        double D = 0.0;
        for (int64_t u = 0; u < V; ++u)
            if (outdeg[u] == 0) D += rank[u];
        for (int64_t u = 0; u < V; ++u)
            contrib[u] = outdeg[u] ? rank[u] / (double)outdeg[u] : 0.0;
        for (int32_t s = 0; s < k; ++s) {
            #pragma omp parallel for schedule(dynamic, 1024)
            for (int64_t i = row_base[s]; i < row_base[s + 1]; ++i) {
                double acc = 0.0;
                for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += contrib[col[e]];
                interm[i] = acc;
            }
        }
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t lo = b * B, hi = lo + B < V ? lo + B : V;
            for (int64_t v = lo; v < hi; ++v) out[v] = 0.0;
            for (int32_t s = 0; s < k; ++s) {
                int64_t bs = row_base[s] + block_start[(int64_t)s * (nb + 1) + b];
                int64_t be = row_base[s] + block_start[(int64_t)s * (nb + 1) + b + 1];
                for (int64_t i = bs; i < be; ++i) out[idx_map[i]] += interm[i];
            }
        }
        double r = 0.0;
        for (int64_t v = 0; v < V; ++v) {
            double nv = base + d * (out[v] + D / (double)V);
            r += fabs(nv - rank[v]);
            rank[v] = nv;
        }
        if (resid) resid[t] = r;
    }
    free(contrib); free(interm); free(out);
    return 0;
}

/*
 * Label propagation, synchronous passes (Table IV's application; min-label
 * connected components): L'[v] = min(L[v], min over in-neighbours u of L[u]).
 * Passes repeat until one changes no label, or max_passes.  `labels` holds
 * the initial labels and receives the final ones.  changes[p] records the
 * number of labels pass p changed (the last recorded pass changed none unless
 * max_passes stopped it).  Returns the number of passes run, or -1.
 */
int64_t orc_label_propagation(int64_t V, const int64_t *offsets, const int32_t *src,
                              int32_t *labels, int64_t max_passes, int64_t *changes) {
    int32_t *next = (int32_t *)malloc((size_t)(V > 0 ? V : 1) * sizeof(int32_t));
    if (!next) return -1;
    int64_t p = 0;
    while (p < max_passes) {
        int64_t changed = 0;
        #pragma omp parallel for schedule(dynamic, 1024) reduction(+:changed)
        for (int64_t v = 0; v < V; ++v) {
            int32_t m = labels[v];
            for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e)
                if (labels[src[e]] < m) m = labels[src[e]];
            next[v] = m;
            changed += (m != labels[v]);
        }
        memcpy(labels, next, (size_t)V * sizeof(int32_t));
        if (changes) changes[p] = changed;
        ++p;
        if (changed == 0) break;
    }
    free(next);
    return p;
}

/*
 * Batched personalised PageRank, FP64, plain definition.  J columns; column j
 * teleports to vertex seeds[j].  With T[v][j] = [v == seeds[j]]:
 *   R_0 = T
 *   D_j = sum over u with outdeg(u) = 0 of R[u][j]
 *   R'[v][j] = (1-d) T[v][j] + d ( sum_{u -> v} R[u][j] / outdeg(u) + D_j T[v][j] )
 * (dangling mass returns to the column's seed).  R is row-major [V][J].
 */
int orc_ppr(int64_t V, const int64_t *offsets, const int32_t *src, int32_t J,
            const int32_t *seeds, int32_t iters, double d, double *R) {
    int64_t *outdeg = (int64_t *)malloc((size_t)(V > 0 ? V : 1) * sizeof(int64_t));
    double *C = (double *)malloc((size_t)(V > 0 ? V : 1) * J * sizeof(double));
    double *N = (double *)malloc((size_t)(V > 0 ? V : 1) * J * sizeof(double));
    double *D = (double *)malloc((size_t)J * sizeof(double));
    if (!outdeg || !C || !N || !D) { free(outdeg); free(C); free(N); free(D); return -1; }
    orc_out_degree(V, offsets, src, outdeg);
    for (int64_t i = 0; i < V * J; ++i) R[i] = 0.0;
    for (int32_t j = 0; j < J; ++j) R[(int64_t)seeds[j] * J + j] = 1.0;
    for (int32_t t = 0; t < iters; ++t) {
        for (int32_t j = 0; j < J; ++j) D[j] = 0.0;
        for (int64_t u = 0; u < V; ++u)
            if (outdeg[u] == 0)
                for (int32_t j = 0; j < J; ++j) D[j] += R[u * J + j];
        #pragma omp parallel for schedule(static)
        for (int64_t u = 0; u < V; ++u)
            for (int32_t j = 0; j < J; ++j)
                C[u * J + j] = outdeg[u] ? R[u * J + j] / (double)outdeg[u] : 0.0;
        #pragma omp parallel for schedule(dynamic, 256)
        for (int64_t v = 0; v < V; ++v) {
            double *row = N + v * J;
            for (int32_t j = 0; j < J; ++j) row[j] = 0.0;
            for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
                const double *c = C + (int64_t)src[e] * J;
                for (int32_t j = 0; j < J; ++j) row[j] += c[j];
            }
            for (int32_t j = 0; j < J; ++j) row[j] = d * row[j];
        }
        for (int32_t j = 0; j < J; ++j) {
            int64_t s = seeds[j];
            N[s * J + j] += (1.0 - d) + d * D[j];
        }
        memcpy(R, N, (size_t)V * J * sizeof(double));
    }
    free(outdeg); free(C); free(N); free(D);
    return 0;
}

/*
 * Collaborative filtering by gradient descent (Table III's application),
 * FP64.  Loss 1/2 sum (r_ui - p_u.q_i)^2 + lambda/2 (sum |p_u|^2 + sum |q_i|^2).
 * One sweep, Jacobi (both sides from the old P, Q):
 *   e_ui = r_ui - p_u . q_i
 *   g_u  = (1/deg u) sum_{i in N(u)} e_ui q_i ;   p_u += step (g_u - lambda p_u)
 *   g_i  = (1/deg i) sum_{u in N(i)} e_ui p_u ;   q_i += step (g_i - lambda q_i)
 * The per-vertex sums run left to right in each side's CSR order.  The user
 * side reads (uoff, uitem, urate); the item side (ioff, iuser, irate).
 * sse_out receives sum e_ui^2 over the user-side CSR, from the old P, Q.
 */
int orc_cf_sweep(int64_t U, int64_t I, int32_t K, const int64_t *uoff,
                 const int32_t *uitem, const uint8_t *urate, const int64_t *ioff,
                 const int32_t *iuser, const uint8_t *irate, double lambda,
                 double step, double *P, double *Q, double *sse_out) {
    if (K < 1 || K > 256) return -1;
    double *P2 = (double *)malloc((size_t)U * K * sizeof(double));
    double *Q2 = (double *)malloc((size_t)I * K * sizeof(double));
    double *sse_u = (double *)malloc((size_t)U * sizeof(double));
    if (!P2 || !Q2 || !sse_u) { free(P2); free(Q2); free(sse_u); return -1; }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t u = 0; u < U; ++u) {
        double sse = 0.0;
        double g[256];
        const double *p = P + u * K;
        for (int32_t k = 0; k < K; ++k) g[k] = 0.0;
        int64_t deg = uoff[u + 1] - uoff[u];
        for (int64_t e = uoff[u]; e < uoff[u + 1]; ++e) {
            const double *q = Q + (int64_t)uitem[e] * K;
            double dot = 0.0;
            for (int32_t k = 0; k < K; ++k) dot += p[k] * q[k];
            double err = (double)urate[e] - dot;
            sse += err * err;
            for (int32_t k = 0; k < K; ++k) g[k] += err * q[k];
        }
        for (int32_t k = 0; k < K; ++k) {
            double gk = deg ? g[k] / (double)deg : 0.0;
            P2[u * K + k] = p[k] + step * (gk - lambda * p[k]);
        }
        sse_u[u] = sse;
    }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < I; ++i) {
        double g[256];
        const double *q = Q + i * K;
        for (int32_t k = 0; k < K; ++k) g[k] = 0.0;
        int64_t deg = ioff[i + 1] - ioff[i];
        for (int64_t e = ioff[i]; e < ioff[i + 1]; ++e) {
            const double *p = P + (int64_t)iuser[e] * K;
            double dot = 0.0;
            for (int32_t k = 0; k < K; ++k) dot += p[k] * q[k];
            double err = (double)irate[e] - dot;
            for (int32_t k = 0; k < K; ++k) g[k] += err * p[k];
        }
        for (int32_t k = 0; k < K; ++k) {
            double gk = deg ? g[k] / (double)deg : 0.0;
            Q2[i * K + k] = q[k] + step * (gk - lambda * q[k]);
        }
    }
    memcpy(P, P2, (size_t)U * K * sizeof(double));
    memcpy(Q, Q2, (size_t)I * K * sizeof(double));
    double sse = 0.0;
    for (int64_t u = 0; u < U; ++u) sse += sse_u[u];
    free(P2); free(Q2); free(sse_u);
    if (sse_out) *sse_out = sse;
    return 0;
}

/*
 * Out-edge CSR of an in-edge CSR by counting: out_off[u+1] - out_off[u] =
 * out-degree of u; the edges u -> v are placed in the order the in-edge CSR
 * lists them (rows v ascending), so each out-row lists its destinations in
 * ascending order.  out_off: int64[V+1], out_dst: int32[E].
 */
int orc_out_csr(int64_t V, const int64_t *offsets, const int32_t *src,
                int64_t *out_off, int32_t *out_dst) {
    int64_t *next = (int64_t *)malloc((size_t)(V > 0 ? V : 1) * sizeof(int64_t));
    if (!next) return -1;
    for (int64_t u = 0; u <= V; ++u) out_off[u] = 0;
    for (int64_t e = 0; e < offsets[V]; ++e) out_off[src[e] + 1]++;
    for (int64_t u = 0; u < V; ++u) out_off[u + 1] += out_off[u];
    for (int64_t u = 0; u < V; ++u) next[u] = out_off[u];
    for (int64_t v = 0; v < V; ++v)
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) out_dst[next[src[e]]++] = (int32_t)v;
    free(next);
    return 0;
}

/*
 * Betweenness-centrality dependencies of one source (the BC of Table V, run
 * from 12 sources; Brandes' algorithm, which the Ligra BC the paper extends
 * follows).  The graph is an OUT-edge CSR (out_off, out_dst): row u lists the
 * w of the edges u -> w.
 *   1. BFS from s over out-edges in FIFO order: level[s] = 0, sigma[s] = 1; for
 *      u taken from the queue and each w in row u: an unvisited w gets
 *      level[u] + 1 and joins the queue; if level[w] = level[u] + 1 then
 *      sigma[w] += sigma[u] (the number of shortest s-w paths).
 *   2. In reverse BFS order: delta[u] = sum over w in row u with
 *      level[w] = level[u] + 1 of sigma[u] / sigma[w] * (1 + delta[w])
 *      (left to right in the row).
 * Unreached vertices get level -1, sigma 0, delta 0.  The centrality of v
 * from a set of sources is the sum of delta over the sources other than v.
 * Returns the number of levels (the largest level + 1), or -1.
 */
int32_t orc_bc_source(int64_t V, const int64_t *out_off, const int32_t *out_dst, int32_t s,
                      int32_t *level, double *sigma, double *delta) {
    int32_t *queue = (int32_t *)malloc((size_t)(V > 0 ? V : 1) * sizeof(int32_t));
    if (!queue || s < 0 || s >= V) { free(queue); return -1; }
    for (int64_t v = 0; v < V; ++v) { level[v] = -1; sigma[v] = 0.0; delta[v] = 0.0; }
    int64_t head = 0, tail = 0;
    level[s] = 0;
    sigma[s] = 1.0;
    queue[tail++] = s;
    while (head < tail) {
        const int32_t u = queue[head++];
        for (int64_t e = out_off[u]; e < out_off[u + 1]; ++e) {
            const int32_t w = out_dst[e];
            if (level[w] < 0) { level[w] = level[u] + 1; queue[tail++] = w; }
            if (level[w] == level[u] + 1) sigma[w] += sigma[u];
        }
    }
    int32_t depth = 0;
    for (int64_t i = tail - 1; i >= 0; --i) {
        const int32_t u = queue[i];
        if (level[u] + 1 > depth) depth = level[u] + 1;
        double acc = 0.0;
        for (int64_t e = out_off[u]; e < out_off[u + 1]; ++e) {
            const int32_t w = out_dst[e];
            if (level[w] == level[u] + 1) acc += sigma[u] / sigma[w] * (1.0 + delta[w]);
        }
        delta[u] = acc;
    }
    free(queue);
    return depth;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
