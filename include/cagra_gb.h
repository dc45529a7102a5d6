/*
 * cagra_gb — C ABI of the GB300 (sm_103a) implementation of the segmented
 * pull gather of "Making Caches Work for Graph Analytics" (Cagra,
 * arXiv 1608.01362): CSR segmenting (Section III), frequency-based
 * clustering (Section V) and the applications built on them.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Graphs are in-edge CSR (Section II-A): row v of (offsets, src) lists the
 *    sources u of the edges u -> v.  offsets has V+1 entries (int64), src has
 *    E entries (int32, each in [0, V)).  V < 2^31, E < 2^31.
 *  - Every pointer argument named dev_* or documented "device" is a device
 *    pointer owned by the CALLER (allocated, e.g., by PyTorch) unless stated
 *    otherwise; "host" pointers are ordinary host memory.  Opaque handles
 *    (cg_segmented, cg_plain) are owned by the LIBRARY: *_create / build
 *    allocates, *_destroy frees.
 *  - Every call is asynchronous on the given stream and returns an int
 *    status: CG_OK (0) or a negative CG_ERR_* code.  Argument checks happen
 *    on the host before anything is enqueued; on error nothing is enqueued
 *    and cg_last_error_message() (thread-local) explains.  Calls that must
 *    read a device result on the host (noted below) synchronize the stream.
 *  - No entry point spins on device flags; no kernel waits on another.
 *  - Handles are bound to the device that was current when they were built;
 *    use them with that device current.
 */
#ifndef CAGRA_GB_H
#define CAGRA_GB_H

#include <stdint.h>
#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define CG_OK 0
#define CG_ERR_INVALID_ARG (-1)
#define CG_ERR_OOM (-2)
#define CG_ERR_CUDA (-3)
#define CG_ERR_TIMEOUT (-4)
#define CG_ERR_UNSUPPORTED (-5)

/* Static text for a status code. */
const char *cg_status_string(int status);
/* Text of the last error raised on the calling thread ("" if none). */
const char *cg_last_error_message(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int cg_version(void);

/* ---------------------------------------------------------------- degrees */

/*
 * Out-degree of every vertex (the `degree` array of Algorithm 1): the number
 * of entries of src equal to u.  dev_src: int32[E]; dev_outdeg: int32[V],
 * overwritten.  Errors: CG_ERR_INVALID_ARG on V < 1, E < 0 or a null pointer
 * with E > 0.
 */
int cg_out_degree(const int32_t *dev_src, int64_t E, int32_t V,
                  int32_t *dev_outdeg, cudaStream_t stream);

/*
 * Reciprocal out-degree (Section VI-B's reciprocal optimisation, Algorithm
 * 5's contrib = rank / outDegree): inv[u] = 1/outdeg[u] in FP32, 0 for a
 * dangling vertex (outdeg 0).  dev_outdeg: int32[V]; dev_inv: float[V].
 */
int cg_inv_outdeg(const int32_t *dev_outdeg, int32_t V, float *dev_inv,
                  cudaStream_t stream);

/* ---------------------------------------------------------------- clustering */

/*
 * Frequency-based clustering (Section V): a stable sort of the vertices on a
 * degree key, hottest first.  mode 0: key = out-degree; mode 1: key =
 * floor(out-degree / max(1, floor(E/V))) (out-degree over the average-degree
 * threshold).  Vertices with equal keys keep their ascending-ID order.
 * dev_outdeg: int32[V] (from cg_out_degree); outputs dev_new_of_old and
 * dev_old_of_new: int32[V], each the inverse of the other.  Bit-exact and
 * deterministic.  Uses stream-ordered scratch (cudaMallocAsync) of about
 * 16 V bytes, freed before return (CG_ERR_OOM if it cannot be had).
 */
int cg_cluster(const int32_t *dev_outdeg, int32_t V, int64_t E, int32_t mode,
               int32_t *dev_new_of_old, int32_t *dev_old_of_new,
               cudaStream_t stream);

/*
 * Renumber an in-edge CSR with a clustering permutation (Section V: the map
 * updates the vertex index in G.edgeArray): new row n is old row
 * old_of_new[n], each source u replaced by new_of_old[u], in-row order kept.
 * Outputs dev_out_offsets: int64[V+1], dev_out_src: int32[E] (must not alias
 * the inputs).  Scratch: 8 (V+1) bytes, stream-ordered.
 */
int cg_relabel_csr(const int64_t *dev_offsets, const int32_t *dev_src,
                   int32_t V, int64_t E, const int32_t *dev_new_of_old,
                   const int32_t *dev_old_of_new, int64_t *dev_out_offsets,
                   int32_t *dev_out_src, cudaStream_t stream);

/*
 * Gather of 4-byte values through an index: out[i] = in[idx[i]] for
 * i in [0, n) (0 where idx[i] is outside [0, n_in)).  Used to carry vertex
 * data between the original and the clustered numbering (Section V keeps
 * both directions of the map): with idx = new_of_old it returns a vector in
 * original IDs from one in clustered IDs.  in/out must not alias.
 */
int cg_permute4(const void *dev_in, int64_t n_in, const int32_t *dev_idx,
                int64_t n, void *dev_out, cudaStream_t stream);

/* The same gather for 8-byte values (FP64 results such as betweenness
 * centrality); both buffers 8-byte aligned. */
int cg_permute8(const void *dev_in, int64_t n_in, const int32_t *dev_idx,
                int64_t n, void *dev_out, cudaStream_t stream);

/*
 * The same gather for rows of row_bytes bytes (a positive multiple of 16;
 * both buffers 16-byte aligned): row i of dev_out = row idx[i] of dev_in
 * (zeros where idx[i] is outside [0, n_in)).  Carries per-vertex rows, such
 * as the 64 ranks per vertex of the batched personalised PageRank, between
 * numberings.  in/out must not alias.
 */
int cg_permute_rows(const void *dev_in, int64_t n_in, int32_t row_bytes,
                    const int32_t *dev_idx, int64_t n, void *dev_out, cudaStream_t stream);

/* ---------------------------------------------------------------- segmenting */

typedef struct cg_segmented cg_segmented;

typedef struct {
  int32_t V;             /* vertices */
  int64_t E;             /* edges */
  int32_t num_segments;  /* k */
  int32_t merge_block;   /* B: destinations per merge block */
  int32_t num_blocks;    /* ceil(V / B) */
  int64_t rows;          /* total subgraph rows = sum_s |dst(s)| = q V */
  double q;              /* expansion factor rows / V (Section III-D) */
  int64_t device_bytes;  /* device memory held by the handle */
  int64_t gather_tiles;  /* 256-edge chunks of one segment-processing pass */
  int32_t table_vertices; /* shared-memory table entries per staged block */
  int32_t ctas_per_sm;   /* staged-gather blocks per SM */
  int32_t gather_threads; /* threads per staged-gather block */
  int32_t staged_segments; /* leading segments served from shared memory */
  int64_t staged_edges;  /* edges of those segments */
  int32_t gather_overlap; /* warps per block serving the L1/L2 segments inside the
                             staged launch (0: a launch of their own) */
  int32_t affine_segments; /* segments after the staged head served from shared memory
                              one block per segment (pr_set_gather_affine) */
  int64_t affine_edges;  /* edges of those segments */
} cg_segmented_info;

/*
 * Preprocessing of Algorithm 2 (Section III-A).  Sources are split into k
 * contiguous ranges [bounds[s], bounds[s+1]); host_bounds (host int64[k+1],
 * bounds[0] = 0, bounds[k] = V, non-decreasing) may be NULL for the paper's
 * uniform split bounds[s] = min(s N, V), N = ceil(V/k).  Subgraph s keeps
 * every in-edge whose source lies in segment s, grouped by destination in
 * the parent's row order, parent edge order kept inside a row; it gets an
 * idxMap (local row -> global destination) and the block indices of the
 * cache-aware merge for blocks of merge_block destinations (Algorithm 4).
 * The handle also owns the intermediate buffers (intermBuf) and the tiling
 * of the gather.  Inputs: device CSR as in the conventions; 1 <= k <= 1024;
 * 1 <= merge_block <= 6144 (a merge block's accumulator lives in one warp's
 * share of shared memory; 512 is a good default).  The call synchronizes the stream (it reads
 * segment sizes on the host).  Errors: CG_ERR_INVALID_ARG, CG_ERR_OOM,
 * CG_ERR_CUDA.  Empty segments are legal.
 */
int pr_build_segments(const int64_t *dev_offsets, const int32_t *dev_src,
                      int32_t V, int64_t E, int32_t num_segments,
                      const int64_t *host_bounds, int32_t merge_block,
                      cg_segmented **out, cudaStream_t stream);

/* Sizes of a segmented graph (host struct, no device work). */
int cg_segmented_get_info(const cg_segmented *seg, cg_segmented_info *info);

/*
 * The expansion factor of Section III-D alone: *q_rows_total = the subgraph
 * rows summed over the segments (each segment's distinct destinations),
 * *q = rows / V (0 for V = 0), *device_bytes = device memory the handle
 * holds.  Any output pointer may be NULL.  Host only, no device work;
 * CG_ERR_INVALID_ARG on a NULL handle.
 */
int cg_segmented_stats(const cg_segmented *seg, int64_t *q_rows_total, double *q,
                       size_t *device_bytes);

/*
 * Segment sizes for this GPU (Section III-D's segment-size choice, re-derived
 * for an SM's shared memory and the L2): after frequency-based clustering the
 * hottest sources come first, so the vertex range is cut into segments of
 * `smem_vertices` sources (-1: the gather's shared-table capacity at one
 * block per SM) for as long as such a segment still carries at least
 * `min_avg_degree` out-edges per vertex, i.e. enough reads to repay staging
 * it on chip; the colder rest is cut into segments of at most
 * `max_global_vertices` sources, served through L1/L2 (<= 0: as many 4-byte
 * source values as fill half of this GPU's L2, from its device properties).
 * dev_outdeg: int32[V]
 * of the (clustered) graph.  Writes k+1 bounds to host_bounds (capacity
 * k_max+1) and k to *k_out.  Synchronizes (reads the degrees on the host).
 */
int pr_plan_bounds(const int32_t *dev_outdeg, int32_t V, int32_t smem_vertices,
                   double min_avg_degree, int32_t max_global_vertices,
                   int32_t k_max, int64_t *host_bounds, int32_t *k_out,
                   cudaStream_t stream);

/*
 * Launch shape of the segment-processing gather of `seg`.  The leading
 * segments of at most `table_vertices` sources (-1: as many as fit in shared
 * memory at `ctas_per_sm` blocks of `threads` threads per SM; 0: none) that
 * carry at least 4 edges per source are "staged": a block copies the
 * segment's source values into shared memory and serves every read of the
 * segment from there.  The other segments are read through L1/L2 by a
 * second launch (1024 threads, 2 blocks per SM, no shared memory).  threads:
 * 512 or 1024; ctas_per_sm <= 1024/threads (the staged kernel holds 64
 * registers per thread): 1 at 1024 threads, 1 or 2 at 512.  Results do not
 * depend on it; CG_ERR_INVALID_ARG otherwise (the previous shape stays).
 * Default after pr_build_segments: 1024, 1, -1.  Synchronizes the stream.
 */
int pr_set_gather_config(cg_segmented *seg, int32_t threads, int32_t ctas_per_sm,
                         int32_t table_vertices, cudaStream_t stream);

/*
 * Overlap of the two kinds of segment processing (Algorithm 3) inside one
 * launch.  cached_warps > 0: one 1024-thread block per SM; warps
 * [0, 32 - cached_warps) of each block work through the staged segments
 * (shared-memory tables), the other cached_warps warps through the L1/L2
 * segments from a chunk queue, and the staged warps join that queue when
 * their own work runs out, so the cold segments' random L2 reads proceed
 * while the staged warps read shared memory.  0 (the default): the staged and
 * the L1/L2 segments get a launch each.  cached_warps in [0, 24]; needs the
 * 1024-thread, 1-block-per-SM shape (pr_set_gather_config) and takes effect
 * while the plan has both kinds of segment.  The row sums do not depend on it
 * (each chunk is summed the same way whichever warp takes it).
 * pr_set_gather_config keeps the setting.  Synchronizes the stream.
 */
int pr_set_gather_overlap(cg_segmented *seg, int32_t cached_warps, cudaStream_t stream);

/*
 * Segment-affine staging of the cold segments (the nested form of two-level
 * segmenting, Section III-B's "smaller segments" in parallel).  With
 * head_min_avg_degree > 0, the leading segments that fit the shared table and
 * carry at least max(4, head_min_avg_degree) edges per source keep the staged
 * schedule (every block sweeps them); the table-fitting segments after them
 * (e.g. the cold source range cut into table-sized segments by pr_plan_bounds
 * with max_global_vertices = the table capacity) are also served from shared
 * memory, but each by ONE block, which takes whole segments from a counter,
 * stages the segment's table once and streams all its edges.  Sources of the
 * cold range are read once per iteration into shared memory instead of once
 * per edge from L2, at the price of more subgraph rows (q) for the merge.
 * 0 turns it off.  Needs the 1024-thread, 1-block-per-SM shape and no overlap
 * (CG_ERR_INVALID_ARG otherwise; the previous configuration stays).
 * Synchronizes.
 */
int pr_set_gather_affine(cg_segmented *seg, double head_min_avg_degree, cudaStream_t stream);

/* Shared-table capacity (entries) of the gather at ctas_per_sm blocks/SM. */
int pr_gather_table_capacity(int32_t ctas_per_sm);

/*
 * Copy the segmented structure out in its canonical flat layout (the layout
 * the FP64 oracle also builds):
 *   host_bounds    int64[k+1]  source range of each segment
 *   host_row_base  int64[k+1]  first subgraph row of each segment
 *   host_edge_base int64[k+1]  first edge of each segment
 *   dev_row_ptr    int64[rows+1] first edge of each subgraph row
 *   dev_col        int32[E]     global source of each edge
 *   dev_idx_map    int32[rows]  global destination of each subgraph row
 *   dev_block_start int32[k*(num_blocks+1)] local row (row - row_base[s]) of
 *                  segment s where block b's destinations begin
 * Any pointer may be NULL to skip that array.  Synchronizes the stream.
 */
int cg_segmented_export(const cg_segmented *seg, int64_t *host_bounds,
                        int64_t *host_row_base, int64_t *host_edge_base,
                        int64_t *dev_row_ptr, int32_t *dev_col,
                        int32_t *dev_idx_map, int32_t *dev_block_start,
                        cudaStream_t stream);

/* Free a segmented graph (synchronizes the device first).  NULL is a no-op. */
int cg_segmented_destroy(cg_segmented *seg);

#define CG_OP_SUM_F32 0
#define CG_OP_MIN_I32 1

/*
 * Parallel segment processing alone (Algorithm 3, Section III-B): for every
 * subgraph row i, interm[i] = op over the row's edges of x[col[e]] (SUM_F32:
 * FP32 sum; MIN_I32: int32 minimum).  Subgraphs are processed in segment
 * order; no atomics.  dev_x: float[V] or int32[V]; dev_interm: rows entries
 * of the same type (caller-owned), or NULL for the handle's own intermBuf
 * (the buffer pr_merge_update reads).
 */
int cg_seg_gather(const cg_segmented *seg, int32_t op, const void *dev_x,
                  void *dev_interm, cudaStream_t stream);

/*
 * The same pass split into its launches, for callers that time or overlap
 * them: phases is a bit mask of 1 = the shared-memory (staged) segments,
 * 2 = the segments read through L1/L2, 4 = the carry fix-up that completes
 * rows spanning chunks.  The three must all run, in this order, before the
 * intermBuf is complete; cg_seg_gather runs all of them.
 */
int cg_seg_gather_phases(const cg_segmented *seg, int32_t op, const void *dev_x,
                         void *dev_interm, int32_t phases, cudaStream_t stream);

/*
 * Cache-aware merge alone (Algorithm 4, Section III-C): for each block of
 * merge_block destinations (one warp per block, its accumulator in shared
 * memory), out[v] = identity (0 / INT32_MAX), then for each segment in
 * ascending order, for its rows i in the block,
 * out[idx_map[i]] = op(out[idx_map[i]], interm[i]).  dev_interm: rows
 * entries; dev_out: V entries.
 */
int merge(const cg_segmented *seg, int32_t op, const void *dev_interm,
          void *dev_out, cudaStream_t stream);

/* ---------------------------------------------------------------- PageRank */

/*
 * PageRank state of Algorithm 5 at r_0 = 1/V: rank[v] = 1/V,
 * contrib[v] = rank[v] * inv[v], and *dev_dangling = sum of rank over the
 * vertices with inv = 0 (FP64).  dev_inv: float[V]; outputs float[V] and one
 * device double.
 */
int pr_init(const float *dev_inv, int32_t V, float *dev_rank,
            float *dev_contrib, double *dev_dangling, cudaStream_t stream);

/*
 * PageRank state for a given rank vector (Algorithm 5's contrib, with the
 * reciprocal degree): contrib[v] = rank[v] * inv[v] and *dev_dangling = sum
 * of rank over the vertices with inv = 0 (FP64, fixed reduction order).
 * Lets a solve start from any caller-supplied rank vector.
 */
int pr_contrib(const float *dev_inv, const float *dev_rank, int32_t V,
               float *dev_contrib, double *dev_dangling, cudaStream_t stream);

/*
 * `iterations` PageRank iterations through the segmented graph: per
 * iteration, Algorithm 3's gather of contrib over every subgraph, then
 * Algorithm 4's blocked merge fused with the vertex update (normalised form,
 * uniform dangling redistribution):
 *   rank'[v]    = (1-d)/V + d (sum_{u->v} contrib[u] + D/V)
 *   contrib'[v] = rank'[v] * inv[v]
 *   D'          = sum of rank' over vertices with inv = 0   (FP64)
 *   resid[t]    = sum_v |rank'[v] - rank[v]|               (FP64)
 * Inputs: dev_inv float[V]; dev_rank_in, dev_contrib_in float[V];
 * *dev_dangling_io (device double) = D of rank_in on entry, D of rank_out on
 * exit.  Outputs: dev_rank_out, dev_contrib_out float[V] (must not alias the
 * inputs); dev_resid: double[iterations] or NULL.  FP32 arithmetic, FP64 only
 * for D and the residual.  Deterministic (fixed reduction order).
 * Iterations > 1 ping-pong through buffers held by the handle.
 */
int pr_iterate(const cg_segmented *seg, const float *dev_inv,
               const float *dev_rank_in, const float *dev_contrib_in,
               float *dev_rank_out, float *dev_contrib_out, double damping,
               int32_t iterations, double *dev_dangling_io, double *dev_resid,
               cudaStream_t stream);

/*
 * One iteration's cache-aware merge fused with the vertex update (Algorithm 4
 * then Algorithm 5's VertexUpdate), reading the handle's intermBuf as left by
 * cg_seg_gather(seg, CG_OP_SUM_F32, contrib, NULL): the second half of one
 * pr_iterate iteration.  *dev_D_in = dangling mass of rank_in; *dev_D_out
 * receives that of rank_out; *dev_resid_out (may be NULL) the FP64 L1
 * residual.  dev_D_in may equal dev_D_out.
 */
int pr_merge_update(const cg_segmented *seg, const float *dev_inv,
                    const float *dev_rank_in, float *dev_rank_out,
                    float *dev_contrib_out, double damping, const double *dev_D_in,
                    double *dev_D_out, double *dev_resid_out, cudaStream_t stream);

/*
 * Personalised PageRank, one vector (the personalised form of the PageRank
 * application; the paper runs the uniform form): the teleport and the
 * dangling mass return to one seed vertex instead of spreading over all V,
 *   rank'[v] = d sum_{u->v} contrib[u] + [v == seed] ((1-d) + d D).
 * pr_init_ppr writes the start state rank = one-hot at the seed, contrib =
 * rank * inv, *dev_dangling = 1 if the seed has no out-edges, else 0.
 * pr_iterate_ppr runs `iterations` of it through the segmented graph with
 * the same arguments, buffers and FP64 reductions as pr_iterate.  seed must
 * be in [0, V) (CG_ERR_INVALID_ARG otherwise).
 */
int pr_init_ppr(const float *dev_inv, int32_t V, int32_t seed, float *dev_rank,
                float *dev_contrib, double *dev_dangling, cudaStream_t stream);
int pr_iterate_ppr(const cg_segmented *seg, const float *dev_inv,
                   const float *dev_rank_in, const float *dev_contrib_in,
                   float *dev_rank_out, float *dev_contrib_out, double damping,
                   int32_t iterations, int32_t seed, double *dev_dangling_io,
                   double *dev_resid, cudaStream_t stream);

/* The plain pull baseline (Algorithm 1 without segmenting). */
typedef struct cg_plain cg_plain;

/*
 * Analyse an in-edge CSR for the plain pull kernel (work tiling over rows +
 * edges) and allocate its work buffers.  The CSR arrays are NOT copied: they
 * must stay valid and unchanged while the handle is used.  Synchronizes.
 */
int pr_plain_create(const int64_t *dev_offsets, const int32_t *dev_src,
                    int32_t V, int64_t E, cg_plain **out, cudaStream_t stream);
int pr_plain_destroy(cg_plain *plain);

/*
 * Same iteration and arguments as pr_iterate, computed by the plain pull
 * gather of Algorithm 1 over the whole CSR (random reads over all of
 * contrib), followed by the vertex update.  probe != 0 is the paper's
 * "lower bound" measurement program (Section I, Fig. 1): every gathered read
 * goes to contrib[0] instead of contrib[src] while the edge stream is read
 * as usual; its result is not PageRank.
 */
int pr_iterate_plain(const cg_plain *plain, const float *dev_inv,
                     const float *dev_rank_in, const float *dev_contrib_in,
                     float *dev_rank_out, float *dev_contrib_out,
                     double damping, int32_t iterations,
                     double *dev_dangling_io, double *dev_resid,
                     int32_t probe, cudaStream_t stream);

/* ---------------------------------------------------- label propagation */

/*
 * One synchronous label-propagation pass over the segmented graph (the LP
 * application of Section VI, Table IV; min-label connected components):
 * L'[v] = min(L[v], min over the in-neighbours u of v of L[u]), computed as
 * Algorithm 3's gather with a minimum, Algorithm 4's merge with a minimum and
 * the label update, all in int32 (exact).  For connected components the graph
 * must hold both directions of every edge.  dev_labels_in / dev_labels_out:
 * int32[V] (must not alias).  dev_changed: device int64 receiving the number
 * of labels this pass changed (NULL: a slot of the handle).  host_changed:
 * if non-NULL the call synchronizes the stream and stores that number.
 */
int lp_iterate(const cg_segmented *seg, const int32_t *dev_labels_in,
               int32_t *dev_labels_out, int64_t *dev_changed,
               int64_t *host_changed, cudaStream_t stream);

/*
 * Passes of lp_iterate until one changes no label (or max_passes): labels in
 * place (device int32[V]).  *host_passes = passes run (the last one changed
 * nothing unless max_passes stopped the loop); host_changes (host int64
 * [max_passes], may be NULL) receives each pass's count.  Synchronizes once
 * per pass (the stopping test reads the count).
 */
int lp_run(const cg_segmented *seg, int32_t *dev_labels, int64_t max_passes,
           int64_t *host_passes, int64_t *host_changes, cudaStream_t stream);

/* ------------------------------------------- batched small-graph PageRank */

typedef struct cg_batch cg_batch;

/*
 * Many independent small graphs for one-launch PageRank (the batched form of
 * the segmented gather; the paper has one graph at a time).  Each graph is
 * its own single shared-memory segment: its contrib vector lives in one
 * SM's shared memory for all iterations.  Input: G graphs concatenated as one
 * in-edge CSR -- host_vbase (host int64[G+1], vbase[0] = 0) gives each
 * graph's vertex range, dev_offsets (device int64[V_total+1]) are global edge
 * offsets, dev_src (device int32[E_total]) holds sources LOCAL to their graph
 * (in [0, V_g)).  Every graph has 1..65536 vertices and must fit one block's
 * shared memory (CG_ERR_UNSUPPORTED otherwise).  The arrays are copied into
 * the handle (flagged edges, per-graph out-degrees); synchronizes.
 */
int pr_batch_create(int32_t G, const int64_t *host_vbase, const int64_t *dev_offsets,
                    const int32_t *dev_src, cg_batch **out, cudaStream_t stream);
int pr_batch_destroy(cg_batch *batch);

/* Threads per block of the batched launch (256, 512 or 1024; default 1024). */
int pr_batch_set_threads(cg_batch *batch, int32_t threads);

/*
 * PageRank of every graph of the batch in ONE persistent launch: r_0 = 1/V_g,
 * `iterations` normalised iterations with uniform dangling redistribution
 * (the same arithmetic as pr_iterate on each graph alone).  Graphs are taken
 * largest first by an atomic counter; a block runs all iterations of its
 * graph on chip.  dev_rank: float[V_total] receives the ranks (graph g's at
 * vbase[g]); dev_resid: double[G*iterations] (graph-major) or NULL.  Stream-
 * ordered and capturable in a CUDA graph (a memset and one kernel).
 */
int pr_batch_run(cg_batch *batch, int32_t iterations, double damping, float *dev_rank,
                 double *dev_resid, cudaStream_t stream);

/* The same call as pr_batch_run, under the name of the batched small-graph
 * form: same arguments, same launch, same errors. */
int pr_batched_graphs_run(cg_batch *batch, int32_t iterations, double damping, float *dev_rank,
                          double *dev_resid, cudaStream_t stream);

/* ----------------------------------- batched personalised PageRank (64) */

typedef struct cg_ppr cg_ppr;

/*
 * 64 personalised PageRank vectors advanced together over one segmented
 * graph (the paper computes one vector at a time; this is its gather and
 * merge with 64-wide rows, an SpMM with a dense 64-column operand).  Column j
 * teleports to seed_j and returns its dangling mass there:
 *   R'[v][j] = d sum_{u->v} C[u][j] + [v == seed_j] ((1-d) + d D_j)
 *   C'[v][j] = R'[v][j] * inv[v],  D'_j = sum over inv[v] = 0 of R'[v][j]
 * The state C is held by the handle as BF16: planes = 2 stores hi = bf16(c)
 * and lo = bf16(c - hi) (about 16 significant bits), planes = 1 stores hi
 * only (8 bits, half the gather traffic); sums are FP32, D_j and residuals
 * FP64.  The segmented graph must outlive the handle and stay unchanged.
 * Memory: about rows*256 + V*(256 + 128*planes) + E/128*260 bytes.
 * Synchronizes.
 */
int ppr_batched_create(const cg_segmented *seg, int32_t planes, cg_ppr **out,
                       cudaStream_t stream);
int ppr_batched_destroy(cg_ppr *ppr);

/* Device bytes held by the handle and its number of 128-edge gather chunks. */
int ppr_batched_bytes(const cg_ppr *ppr, int64_t *bytes, int64_t *chunks);

/*
 * Start state: R_0 = one-hot at each column's seed.  host_seeds: host
 * int32[64], each in [0, V) (repeats allowed).  dev_inv: float[V], the
 * reciprocal out-degrees of the segmented graph's vertices.  Synchronizes.
 */
int ppr_batched_init(cg_ppr *ppr, const float *dev_inv, const int32_t *host_seeds,
                     cudaStream_t stream);

/*
 * `iterations` iterations from the handle's current state.  dev_rank_out
 * (float[V][64], row-major: vertex v's 64 values contiguous, or NULL)
 * receives R after the last iteration.  dev_resid (double[64] or NULL; needs
 * iterations >= 2 and dev_rank_out) receives sum_v |R_T[v][j] - R_{T-1}[v][j]|
 * per column.  Stream-ordered; capturable in a CUDA graph.
 */
int ppr_batched_iterate(cg_ppr *ppr, const float *dev_inv, double damping,
                        int32_t iterations, float *dev_rank_out, double *dev_resid,
                        cudaStream_t stream);

/*
 * One iteration's launches selected by `phases` (1 gather, 2 carry fix-up,
 * 4 merge + update, 8 the tensor-core hub block of ppr_batched_attach_dense;
 * 15 = one whole iteration, 7 when no hub block is attached), for timing each
 * launch; phases in [0, 15].  The
 * merge writes R' to dev_rank_out when non-NULL and, when dev_rank_old is
 * given, the per-column L1 distance to it in dev_resid (double[64], may be
 * NULL).
 */
int ppr_batched_step(cg_ppr *ppr, const float *dev_inv, double damping, int32_t phases,
                     const float *dev_rank_old, float *dev_rank_out, double *dev_resid,
                     cudaStream_t stream);

/* ------------------------------------------------ collaborative filtering */

typedef struct cg_bipartite cg_bipartite;

/*
 * Item-major copy of a user-major rating CSR (the other side of the
 * bipartite graph): dev_uoff int64[U+1], dev_uitem int32[R] (items in
 * [0, I)), dev_urate uint8[R] -> dev_ioff int64[I+1], dev_iuser int32[R]
 * (users ascending within each item: a stable sort by item), dev_irate
 * uint8[R].  Out-of-range items give CG_ERR_INVALID_ARG.  Synchronizes.
 */
int cf_transpose(int64_t U, int64_t I, const int64_t *dev_uoff, const int32_t *dev_uitem,
                 const uint8_t *dev_urate, int64_t *dev_ioff, int32_t *dev_iuser,
                 uint8_t *dev_irate, cudaStream_t stream);

/*
 * Collaborative filtering by gradient descent (the CF application of
 * Section VI, Table III; the paper gives no formula, so the loss is
 * 1/2 sum (r_ui - p_u.q_i)^2 + lambda/2 (|P|^2 + |Q|^2) with the
 * degree-averaged gradient).  The rating CSRs of both sides (from
 * cf_transpose) are NOT copied and must stay valid.  K = 16, 32 or 64
 * latent dimensions.  precision: 0 stores P, Q in FP32, 1 in BF16, 2 as
 * BF16 hi + lo pairs (hi = bf16(x), lo = bf16(x - hi), packed in one 32-bit
 * word per entry: a row has the size and alignment of FP32); arithmetic is FP32
 * and the squared-error sum FP64.  The handle owns the factor storage (see
 * cf_set_factors).  Synchronizes.
 */
int cf_create(int64_t U, int64_t I, int32_t K, int32_t precision, const int64_t *dev_uoff,
              const int32_t *dev_uitem, const uint8_t *dev_urate, const int64_t *dev_ioff,
              const int32_t *dev_iuser, const uint8_t *dev_irate, cg_bipartite **out,
              cudaStream_t stream);
int cf_destroy(cg_bipartite *cf);

/* Load the factors (device FP32, row-major P[U][K], Q[I][K]) into the
 * handle's storage format (rounding to BF16 where it stores BF16). */
int cf_set_factors(cg_bipartite *cf, const float *dev_P, const float *dev_Q,
                   cudaStream_t stream);
/* Read the stored factors back as FP32 (either pointer may be NULL). */
int cf_get_factors(const cg_bipartite *cf, float *dev_P, float *dev_Q, cudaStream_t stream);

/*
 * `sweeps` Jacobi sweeps: both sides read the old P, Q;
 *   e_ui = r_ui - p_u . q_i
 *   p_u += step ((1/deg u) sum_{i in N(u)} e_ui q_i - lambda p_u)
 *   q_i += step ((1/deg i) sum_{u in N(i)} e_ui p_u - lambda q_i)
 * (vertices without ratings only decay).  dev_sse: double[sweeps] or NULL;
 * entry t receives sum over ratings of e_ui^2 for the factors entering
 * sweep t.  Stream-ordered; deterministic for a given device.
 */
int cf_sweep(cg_bipartite *cf, int32_t sweeps, double lambda, double step, double *dev_sse,
             cudaStream_t stream);

/* One launch of a sweep (0 user gather + SSE, 1 item gather, 2 user update,
 * 3 item update; a sweep is 0, 1, 2, 3 in that order), for timing. */
int cf_sweep_phase(cg_bipartite *cf, int32_t phase, double lambda, double step,
                   double *dev_sse, cudaStream_t stream);

/* Ratings, gather pieces per side and device bytes of the handle. */
int cf_info(const cg_bipartite *cf, int64_t *ratings, int64_t *user_pieces,
            int64_t *item_pieces, int64_t *bytes);

/* ------------------------------------------------- no device allocation */

/*
 * One plain pull PageRank iteration (the same arithmetic as pr_iterate_plain
 * with iterations = 1 and probe = 0) that allocates no device memory.  The
 * paper has no counterpart: this exists for callers that cannot allocate at
 * call time -- code running inside a memory budget reserved up front, hosts
 * that only let a library touch buffers they registered beforehand, or
 * latency-critical loops that must not risk the synchronisation an
 * allocation can cause.  Such a caller passes its own inputs and outputs
 * (device pointers, as for pr_iterate_plain: in-edge CSR, inv, rank_in,
 * contrib_in -> rank_out, contrib_out; *dev_dangling_io = D of rank_in on
 * entry, D of rank_out on exit; dev_resid: one double or NULL) and the work
 * buffers come from one statically sized device array inside the library,
 * which every GPU that loads the library holds until the process exits (see
 * pr_noalloc_limits for its size).
 *  - Limits: V <= 2^20 vertices and E <= 2^24 edges; larger inputs return
 *    CG_ERR_INVALID_ARG with a message and enqueue nothing.
 *  - The CSR is not validated (validation would need scratch).  The caller
 *    must pass offsets that rise monotonically from offsets[0] = 0 to
 *    offsets[V] = E.  Out-of-range sources are skipped.  Offsets that break
 *    this give unspecified rank values but no out-of-bounds memory access:
 *    the gather clamps every tile's row and edge counts to the tile.
 *  - No cudaMalloc, cudaFree or allocating library routine is called.  The
 *    first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.
 *  - Every call shares the one array and the array keeps the last call's
 *    contents: calls whose executions overlap on the GPU (other streams,
 *    other host threads) race with each other.  Serialise them.
 */
int pr_iterate_plain_noalloc(const int64_t *dev_offsets, const int32_t *dev_src,
                             int32_t V, int64_t E, const float *dev_inv,
                             const float *dev_rank_in, const float *dev_contrib_in,
                             float *dev_rank_out, float *dev_contrib_out,
                             double damping, double *dev_dangling_io,
                             double *dev_resid, cudaStream_t stream);

/*
 * Dense hub block of the batched personalised PageRank on the tensor cores.
 * After frequency-based clustering (Section V) the hottest vertices carry the
 * lowest IDs and the block of the adjacency matrix among vertices [0, h) is
 * dense; its share of the batched gather becomes a contraction Y = A_H C_H
 * (A_H: the 0/1 hub block, row = destination; C_H: the hubs' 64-column
 * contributions in BF16 hi and lo planes), computed with tcgen05.mma (BF16
 * operands, FP32 accumulators in tensor memory) and added by the merge as one
 * more intermBuf row per hub destination.  Not in the paper (it extends the
 * batched form of Algorithm 3).
 *
 * cg_split_hub_block: splits an in-edge CSR (validated; V >= h, h a positive
 * multiple of 128) into the rest (dev_out_offsets int64[V+1], dev_out_src
 * int32[E] capacity: every edge with source or destination >= h, in the input
 * order) and the hub block as a bitmap dev_bits uint32[h][h/32] (bit u of row
 * v set when u -> v, u, v < h; overwritten).  *host_E_rest receives the rest's
 * edge count.  Synchronizes.
 *
 * ppr_batched_attach_dense: attaches such a block to a batched handle built
 * over the rest's segmented graph (same V and vertex numbering).  dev_bits is
 * caller-owned and must stay valid while the handle is used.  From then on
 * ppr_batched_iterate also runs the tensor-core launch (phase 8 of
 * ppr_batched_step: the 64-source chunks of each 128-destination tile that
 * hold an edge are split over up to 8 CTAs of eight expander warps and one
 * MMA/copy warp, two CTAs per SM; the tile's last CTA to finish adds the
 * parts in part order, so the result does not depend on timing), and each
 * merge phase repacks
 * the hubs' contributions into the operand layout.  CG_ERR_UNSUPPORTED on a GPU without
 * tcgen05 (compute capability other than 10.x); CG_ERR_INVALID_ARG on a bad h
 * or a second attach.  A launch whose bounded waits (operand copies, tensor
 * work) give up records a fault; the next step returns CG_ERR_TIMEOUT.
 */
int cg_split_hub_block(const int64_t *dev_in_offsets, const int32_t *dev_in_src, int32_t V,
                       int64_t E, int32_t h, int64_t *dev_out_offsets, int32_t *dev_out_src,
                       uint32_t *dev_bits, int64_t *host_E_rest, cudaStream_t stream);
int ppr_batched_attach_dense(cg_ppr *ppr, int32_t h, const uint32_t *dev_bits,
                             cudaStream_t stream);

/* ------------------------------------------------ betweenness centrality */

/*
 * Transpose of an in-edge CSR: the out-edge CSR, row u listing the w of the
 * edges u -> w in ascending order (a stable radix sort of the edges by
 * source).  dev_in_offsets int64[V+1], dev_in_src int32[E] (validated: offsets
 * monotone from 0 to E, sources in [0, V)); dev_out_offsets int64[V+1] and
 * dev_out_dst int32[E] are overwritten.  Scratch (about 12 E bytes) comes from
 * the stream-ordered allocator.  CG_ERR_INVALID_ARG on a bad CSR or sizes.
 * Synchronizes the stream (validation).
 */
int cg_transpose_csr(const int64_t *dev_in_offsets, const int32_t *dev_in_src, int32_t V,
                     int64_t E, int64_t *dev_out_offsets, int32_t *dev_out_dst,
                     cudaStream_t stream);

/*
 * Betweenness centrality from a set of sources: the BC application of the
 * paper's Table V (12 sources), which tracks an active set of vertices (the
 * VertexSubset / ActiveFrontier of EdgeMap, Section IV), by Brandes'
 * algorithm.  For each source s: a BFS over out-edges gives every vertex's
 * level and sigma[v] = number of shortest s-v paths; then, deepest level
 * first, delta[u] = sum over out-neighbours w one level deeper of
 * sigma[u] / sigma[w] * (1 + delta[w]); bc[v] += delta[v] for v != s.
 *
 * bc_create takes the graph as both an in-edge CSR (dev_in_offsets,
 * dev_in_src: the pull direction) and its out-edge CSR (dev_out_offsets,
 * dev_out_dst, e.g. from cg_transpose_csr: the push direction and the
 * dependency sums); both caller-owned, validated, and read for the handle's
 * lifetime.  The handle (library-owned, about 60 V bytes) holds the
 * per-source state.  CG_ERR_INVALID_ARG on bad sizes or CSRs.  Synchronizes.
 *
 * bc_run: for each of the nsources host vertex IDs (each in [0, V), repeats
 * allowed) in turn, adds its dependencies into dev_bc (FP64[V], caller-owned;
 * zero it before the first call to get the centrality of the whole set).
 * Each BFS level runs push (one thread per out-edge of the frontier, found
 * through a prefix sum of the frontier's degrees; level by compare-and-swap,
 * sigma by FP64 atomic adds) or pull, bottom-up (a merge-path tile gather
 * over the in-edges of the unvisited vertices of sigma on the frontier, 0
 * elsewhere) as the frontier's out-edges times alpha stay below or exceed E.
 * sigma values are integers and exact in FP64 below 2^53, so levels and sigma
 * are the same in any order or direction; delta sums run in a fixed order
 * (deterministic).  Reads a few counts per level on the host: synchronizes
 * the stream.
 *
 * bc_set_direction: alpha >= 0 (default 16; 0 always pushes, a huge value
 * pulls every level with a non-empty frontier).
 *
 * bc_source_state: the last source's levels (int32[V], -1 unreached), sigma
 * and delta (FP64[V]) copied into caller device buffers (any may be NULL),
 * its number of levels and how many ran push and pull (host; may be NULL).
 */
typedef struct cg_bc cg_bc;
int bc_create(const int64_t *dev_in_offsets, const int32_t *dev_in_src,
              const int64_t *dev_out_offsets, const int32_t *dev_out_dst, int32_t V,
              int64_t E, cg_bc **out, cudaStream_t stream);
int bc_destroy(cg_bc *bc);
int bc_set_direction(cg_bc *bc, double alpha);
int bc_run(cg_bc *bc, const int32_t *sources, int32_t nsources, double *dev_bc,
           cudaStream_t stream);
int bc_source_state(const cg_bc *bc, int32_t *dev_level, double *dev_sigma,
                    double *dev_delta, int32_t *depth, int32_t *push_levels,
                    int32_t *pull_levels, cudaStream_t stream);

/* Limits and size of the fixed scratch of pr_iterate_plain_noalloc (host). */
int pr_noalloc_limits(int64_t *max_vertices, int64_t *max_edges,
                      int64_t *scratch_bytes);

#ifdef __cplusplus
}
#endif
#endif /* CAGRA_GB_H */
