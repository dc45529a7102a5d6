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
 */
int orc_pagerank(int64_t V, const int64_t *offsets, const int32_t *src,
                 int32_t iters, double d, double *rank, double *resid) {
    int64_t *outdeg = (int64_t *)malloc((size_t)V * sizeof(int64_t));
    double *contrib = (double *)malloc((size_t)V * sizeof(double));
    double *next = (double *)malloc((size_t)V * sizeof(double));
    if (!outdeg || !contrib || !next) { free(outdeg); free(contrib); free(next); return -1; }
    orc_out_degree(V, offsets, src, outdeg);
    const double base = (1.0 - d) / (double)V;
    for (int32_t t = 0; t < iters; ++t) {
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
            next[v] = base + d * (s + D / (double)V);
        }
        double r = 0.0;
        for (int64_t v = 0; v < V; ++v) r += fabs(next[v] - rank[v]);
        if (resid) resid[t] = r;
        memcpy(rank, next, (size_t)V * sizeof(double));
    }
    free(outdeg); free(contrib); free(next);
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

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
