// The pull gather shared by every application: for every row i of a CSR
// (rows = subgraph rows of the segmented graph, or destinations of the plain
// graph) out[i] = op over the row's edges e of x[col[e]].
//
// Work split (merge-path over rows + edges): the merged sequence of "row
// ends" and "edges" (rows + E items) of every segment is cut into tiles of
// TILE = THREADS * IPT items, so every tile costs the same however skewed the
// row lengths are; tiles never straddle two segments.  The tiles' start
// (row, edge) and segment are computed once per graph.
//
// A persistent grid walks the tiles round-robin (tile t goes to block
// t mod grid), so all blocks move through the segments together, in segment
// order, as Algorithm 3 prescribes.  Each block keeps a shared-memory copy of
// the first `tab_cap` source values of its current segment: a segment no
// larger than that is served entirely from shared memory (the on-chip
// analogue of the paper's cache-sized segment); in a larger segment the
// table holds its hottest head (vertices are clustered hottest-first) and
// the other reads go through L1/L2.  In a tile:
//   1. edges: coalesced streaming reads of col, then the value reads (table
//      or global) into shared memory;
//   2. row ends of the tile's rows into shared memory;
//   3. each thread walks IPT consecutive merged items sequentially, folding
//      edges into its running value and emitting a row at each row end;
//   4. a block-wide segmented scan over the threads' open-row carries gives
//      each thread the part of its first row that earlier threads hold;
//   5. row results are written coalesced; the part of the row still open at
//      the tile's end goes to carry[tile] and is folded in by a small fix-up
//      kernel in tile order.
// Shared arrays indexed by item are padded one word per 32 so the threads'
// strided walks hit distinct banks.  No atomics; deterministic.
#pragma once

#include <vector>

#include "common.cuh"

namespace cg {

struct SumF32 {
  using T = float;
  static __device__ __forceinline__ T identity() { return 0.0f; }
  static __device__ __forceinline__ T op(T a, T b) { return a + b; }
};
struct MinI32 {
  using T = int32_t;
  static __device__ __forceinline__ T identity() { return 0x7FFFFFFF; }
  static __device__ __forceinline__ T op(T a, T b) { return a < b ? a : b; }
};

// Merge-path search: number of rows consumed among the first `diag` merged
// items, given row_end[] relative to the first edge (edge j is consumed
// before row i iff j < row_end[i]).  PADDED reads row_end[i + i/32].
template <bool PADDED, typename RowEndT>
__device__ __forceinline__ int64_t merge_path_search(int64_t diag, const RowEndT* row_end,
                                                     int64_t nrows, int64_t nedges,
                                                     int64_t edge0) {
  int64_t lo = diag - nedges > 0 ? diag - nedges : 0;
  int64_t hi = diag < nrows ? diag : nrows;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t m = PADDED ? mid + (mid >> 5) : mid;
    if ((int64_t)row_end[m] - edge0 <= diag - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int pad32(int p) { return p + (p >> 5); }

// Tile boundaries: tile t lies in segment s = tile_seg[t]; its start is the
// merge-path point at diagonal seg_diag[s] + (t - tile_base[s]) * tile.
template <typename RowEndT>
__global__ void tile_partition_kernel(const RowEndT* __restrict__ row_end, int64_t nrows,
                                      int64_t nedges, int64_t tile, int64_t ntiles, int k,
                                      const int64_t* __restrict__ tile_base,
                                      const int64_t* __restrict__ seg_diag,
                                      int32_t* __restrict__ tile_row,
                                      int32_t* __restrict__ tile_edge,
                                      int32_t* __restrict__ tile_seg) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t d;
    if (t == ntiles) {
      d = nrows + nedges;
    } else {
      int lo = 0, hi = k + 1;  // last s with tile_base[s] <= t (non-empty segments only)
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (tile_base[mid] <= t) lo = mid + 1; else hi = mid;
      }
      const int s = lo - 1;
      tile_seg[t] = s;
      d = seg_diag[s] + (t - tile_base[s]) * tile;
    }
    const int64_t i = merge_path_search<false>(d, row_end, nrows, nedges, 0);
    tile_row[t] = (int32_t)i;
    tile_edge[t] = (int32_t)(d - i);
  }
}

// The persistent gather kernel.  row_end[i] = first edge after row i (global
// edge index); col: global source IDs; seg_lo[s]: first source of segment s;
// seg_tab[s]: how many of its first sources the shared table holds.  PROBE
// sends every read to x[0] (the paper's lower-bound program).
template <class Op, int THREADS, int IPT, bool PROBE, typename RowEndT>
__global__ void __launch_bounds__(THREADS)
gather_kernel(const RowEndT* __restrict__ row_end, const int32_t* __restrict__ col,
              const typename Op::T* __restrict__ x, int32_t nx,
              const int32_t* __restrict__ tile_row, const int32_t* __restrict__ tile_edge,
              const int32_t* __restrict__ tile_seg, int64_t ntiles,
              const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_tab,
              int tab_cap, typename Op::T* __restrict__ out, typename Op::T* __restrict__ carry,
              int32_t* __restrict__ carry_row) {
  using T = typename Op::T;
  constexpr int TILE = THREADS * IPT;
  constexpr int PADT = TILE + TILE / 32;
  constexpr int WARPS = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);       // [tab_cap]
  T* s_val = tab + tab_cap;                      // [PADT] edge values
  int32_t* s_rend = reinterpret_cast<int32_t*>(s_val + PADT);  // [PADT] row ends, then results
  __shared__ T s_wval[WARPS];
  __shared__ int32_t s_wrow[WARPS];
  __shared__ T s_prev_val[THREADS];
  __shared__ int32_t s_prev_row[THREADS];

  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  int cur_seg = -1;
  int32_t lo = 0, tn = 0;

  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int s = tile_seg[t];
    const int32_t r0 = tile_row[t], r1 = tile_row[t + 1];
    const int32_t e0 = tile_edge[t], e1 = tile_edge[t + 1];
    const int nr = r1 - r0, ne = e1 - e0;
    __syncthreads();  // the previous tile is done with every shared array
    if (!PROBE && s != cur_seg) {
      cur_seg = s;
      lo = seg_lo[s];
      tn = seg_tab[s] < tab_cap ? seg_tab[s] : tab_cap;
      for (int i = tid; i < tn; i += THREADS) tab[i] = x[lo + i];
      __syncthreads();
    }

    // 1. edges: stream col, read values (shared table or global)
    {
      int32_t c[IPT];
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        const int j = u * THREADS + tid;
        c[u] = j < ne ? __ldcs(col + e0 + j) : -1;
      }
      T v[IPT];
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        const int32_t cu = c[u];
        if (PROBE) {
          v[u] = cu >= 0 ? __ldg(x) : Op::identity();
        } else {
          const uint32_t off = (uint32_t)(cu - lo);
          if (off < (uint32_t)tn)
            v[u] = tab[off];
          else
            v[u] = (cu >= 0 && cu < nx) ? __ldg(x + cu) : Op::identity();
        }
      }
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        const int j = u * THREADS + tid;
        if (j < ne) s_val[pad32(j)] = v[u];
      }
    }
    // 2. row ends relative to e0 (in [0, ne] for the tile's rows)
    for (int i = tid; i < nr; i += THREADS)
      s_rend[pad32(i)] = (int32_t)((int64_t)row_end[r0 + i] - e0);
    __syncthreads();

    // 3. sequential walk over this thread's merged items
    const int items = nr + ne;
    const int d0 = tid * IPT < items ? tid * IPT : items;
    const int d1 = d0 + IPT < items ? d0 + IPT : items;
    int i = (int)merge_path_search<true, int32_t>(d0, s_rend, nr, ne, 0);
    int j = d0 - i;
    __syncthreads();  // every search is done before row results overwrite s_rend
    const int first_row = i;
    bool emitted = false;
    T first_val = Op::identity();
    T acc = Op::identity();
    for (int d = d0; d < d1; ++d) {
      if (i < nr && s_rend[pad32(i)] <= j) {
        if (!emitted) {
          first_val = acc;
          emitted = true;
        } else {
          reinterpret_cast<T*>(s_rend)[pad32(i)] = acc;
        }
        acc = Op::identity();
        ++i;
      } else {
        acc = Op::op(acc, s_val[pad32(j)]);
        ++j;
      }
    }

    // 4. block segmented inclusive scan of the (open row, value) carries
    int32_t crow = i;
    T cval = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t prow = __shfl_up_sync(0xffffffffu, crow, o);
      const T pval = __shfl_up_sync(0xffffffffu, cval, o);
      if (lane >= o && prow == crow) cval = Op::op(pval, cval);
    }
    if (lane == 31) {
      s_wrow[w] = crow;
      s_wval[w] = cval;
    }
    __syncthreads();
    if (w == 0) {
      int32_t r = lane < WARPS ? s_wrow[lane] : -1;
      T v = lane < WARPS ? s_wval[lane] : Op::identity();
#pragma unroll
      for (int o = 1; o < WARPS; o <<= 1) {
        const int32_t prow = __shfl_up_sync(0xffffffffu, r, o);
        const T pval = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o && prow == r) v = Op::op(pval, v);
      }
      if (lane < WARPS) s_wval[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    if (w > 0 && s_wrow[w - 1] == crow) cval = Op::op(s_wval[w - 1], cval);
    s_prev_row[tid] = crow;
    s_prev_val[tid] = cval;
    __syncthreads();
    if (emitted) {
      T v = first_val;
      if (tid > 0 && s_prev_row[tid - 1] == first_row) v = Op::op(s_prev_val[tid - 1], v);
      reinterpret_cast<T*>(s_rend)[pad32(first_row)] = v;
    }
    __syncthreads();

    // 5. coalesced row results; tile carry for the row open at the tile end
    for (int r = tid; r < nr; r += THREADS)
      out[r0 + r] = reinterpret_cast<T*>(s_rend)[pad32(r)];
    if (tid == THREADS - 1) {
      carry[t] = cval;  // the last thread's inclusive value is the open row's tile part
      carry_row[t] = r0 + crow;
    }
  }
}

// Fold the tile carries into the rows they belong to, in tile order: the
// first tile of each run of tiles carrying the same row sums the run.
template <class Op>
__global__ void carry_fixup_kernel(const typename Op::T* __restrict__ carry,
                                   const int32_t* __restrict__ carry_row, int64_t ntiles,
                                   int64_t nrows, typename Op::T* __restrict__ out) {
  using T = typename Op::T;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = carry_row[t];
    if (r < 0 || r >= nrows) continue;
    if (t > 0 && carry_row[t - 1] == r) continue;
    T s = carry[t];
    for (int64_t u = t + 1; u < ntiles && carry_row[u] == r; ++u) s = Op::op(s, carry[u]);
    out[r] = Op::op(s, out[r]);
  }
}

constexpr int kGatherThreads = 256;
constexpr int kGatherIPT = 8;
constexpr int kGatherTile = kGatherThreads * kGatherIPT;
constexpr int kGatherPadTile = kGatherTile + kGatherTile / 32;
// Static shared memory of gather_kernel (scan scratch), for occupancy sizing.
constexpr int kGatherStaticSmem = kGatherThreads * 8 + 64 + 64;

// Tiling of one gather: per-tile start row / edge / segment, per-segment
// source range and table length, the carry buffers and the launch shape.
struct GatherPlan {
  int64_t nrows = 0, nedges = 0, ntiles = 0, tile = 0;
  int k = 0;
  int32_t* tile_row = nullptr;   // [ntiles+1]
  int32_t* tile_edge = nullptr;  // [ntiles+1]
  int32_t* tile_seg = nullptr;   // [ntiles]
  int32_t* seg_lo = nullptr;     // [k] first source of each segment
  int32_t* seg_tab = nullptr;    // [k] table length of each segment
  void* carry = nullptr;         // [ntiles] 4-byte values
  int32_t* carry_row = nullptr;  // [ntiles]
  std::vector<int64_t> src_bounds;  // host copy [k+1]
  int tab_cap = 0;               // shared table capacity (entries)
  int ctas_per_sm = 2;
  int grid = 0;
};

// Largest table (entries, multiple of 32) that lets `ctas` blocks share an SM.
int gather_table_capacity(int ctas);

// Build a plan (cudaMalloc: the plan lives with its handle).  row_base /
// edge_base / src_bounds: host arrays of k+1 entries (one segment for the
// plain CSR).  Synchronizes the stream.
template <typename RowEndT>
int plan_gather(const RowEndT* row_end, int64_t nrows, int64_t nedges, int k,
                const std::vector<int64_t>& row_base, const std::vector<int64_t>& edge_base,
                const std::vector<int64_t>& src_bounds, int tab_vertices, int ctas_per_sm,
                GatherPlan* p, cudaStream_t s);

// Set the shared table size (-1: the largest that fits ctas_per_sm blocks,
// 0: none) and the blocks per SM; recomputes the per-segment table lengths.
int configure_gather(GatherPlan* p, int tab_vertices, int ctas_per_sm, cudaStream_t s);

void free_plan(GatherPlan* p);
int64_t plan_bytes(const GatherPlan& p);

template <class Op, bool PROBE, typename RowEndT>
int run_gather(const GatherPlan& p, const RowEndT* row_end, const int32_t* col,
               const typename Op::T* x, int32_t nx, typename Op::T* out, cudaStream_t s);

}  // namespace cg
