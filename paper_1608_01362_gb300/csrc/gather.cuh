// The plain pull gather (Algorithm 1) over a caller's CSR: for every row i,
// out[i] = op over the row's edges e of x[col[e]].  The segmented graph uses
// the flagged-edge gather of seg_gather.cuh instead.
//
// Work split (merge-path over rows + edges): the merged sequence of "row
// ends" and "edges" (rows + E items) is cut into tiles of TILE = THREADS *
// IPT items, so every block does the same amount of work however skewed the
// row lengths are.  A tile's start (row, edge) is precomputed once per graph
// (static across iterations).  In a tile:
//   1. edges: coalesced streaming reads of col, then the random reads of x
//      (many independent loads in flight per thread) into shared memory;
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

#include "common.cuh"

namespace cg {

// kExactAnyOrder: the combination gives the same result in any order (and a
// shared-memory atomic can apply it), so a merge need not keep segment order.
struct SumF32 {
  using T = float;
  static constexpr bool kExactAnyOrder = false;  // FP rounding depends on the order
  static __device__ __forceinline__ T identity() { return 0.0f; }
  static __device__ __forceinline__ T op(T a, T b) { return a + b; }
  static __device__ __forceinline__ void atomic_op(T* p, T v) { *p = op(*p, v); }
};
// FP64 sums (betweenness centrality: path counts, which are exact integers in
// any order below 2^53, and dependencies).
struct SumF64 {
  using T = double;
  static constexpr bool kExactAnyOrder = false;
  static __device__ __forceinline__ T identity() { return 0.0; }
  static __device__ __forceinline__ T op(T a, T b) { return a + b; }
  static __device__ __forceinline__ void atomic_op(T* p, T v) { *p = op(*p, v); }
};
struct MinI32 {
  using T = int32_t;
  static constexpr bool kExactAnyOrder = true;
  static __device__ __forceinline__ T identity() { return 0x7FFFFFFF; }
  static __device__ __forceinline__ T op(T a, T b) { return a < b ? a : b; }
  static __device__ __forceinline__ void atomic_op(T* p, T v) { atomicMin(p, v); }
};

// Read-only random load of a gathered vertex value (L1-cached).
template <typename T>
__device__ __forceinline__ T ld_gather(const T* p) { return __ldg(p); }

__device__ __forceinline__ int pad32(int p) { return p + (p >> 5); }

// Merge-path search: number of rows consumed among the first `diag` merged
// items, given row_end[] relative to the first edge (edge j is consumed
// before row i iff j < row_end[i]).
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

// One thread per tile boundary t in [0, ntiles]: (row, edge) at diagonal t*TILE.
template <typename RowEndT>
__global__ void tile_partition_kernel(const RowEndT* __restrict__ row_end, int64_t nrows,
                                      int64_t nedges, int64_t tile, int64_t ntiles,
                                      int32_t* __restrict__ tile_row,
                                      int32_t* __restrict__ tile_edge) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = t * tile;
    if (d > nrows + nedges) d = nrows + nedges;
    const int64_t i = merge_path_search<false>(d, row_end, nrows, nedges, 0);
    tile_row[t] = (int32_t)i;
    tile_edge[t] = (int32_t)(d - i);
  }
}

// The gather tile kernel.  row_end[i] = first edge after row i (global edge
// index); col: global source IDs; PROBE sends every gathered read to x[0].
// MASKED: xmask holds one bit per source; x is read only where the bit is
// set (the identity elsewhere), so a sparse x (a frontier) costs a bit test
// from a small, cache-resident array instead of a value read per edge.
// VIRT: the rows are rows of another CSR (voff, vadj) taken in the order of
// a vertex list vlist (row i = vertex vlist[i]; row_end: their lengths'
// inclusive prefix); each edge's source is read through the list
// (vadj[voff[vlist[i]] + position in the row]) instead of from col, so a
// subset of a graph's rows is gathered without being copied out first.
template <class Op, int THREADS, int IPT, bool PROBE, typename RowEndT, bool MASKED = false,
          bool VIRT = false>
__global__ void __launch_bounds__(THREADS)
gather_tile_kernel(const RowEndT* __restrict__ row_end, const int32_t* __restrict__ col,
                   const typename Op::T* __restrict__ x, int32_t nx,
                   const int32_t* __restrict__ tile_row, const int32_t* __restrict__ tile_edge,
                   typename Op::T* __restrict__ out, typename Op::T* __restrict__ carry,
                   int32_t* __restrict__ carry_row,
                   const uint32_t* __restrict__ xmask = nullptr,
                   const int32_t* __restrict__ vlist = nullptr,
                   const int64_t* __restrict__ voff = nullptr,
                   const int32_t* __restrict__ vadj = nullptr) {
  using T = typename Op::T;
  constexpr int TILE = THREADS * IPT;
  constexpr int WARPS = THREADS / 32;
  constexpr int PADT = TILE + TILE / 32;
  __shared__ T s_val[PADT];
  __shared__ int32_t s_rend[PADT];  // row ends relative to the tile's first edge
  // Row results.  A row emitted during the walk lies wholly inside the
  // emitting thread's items (a row that began in an earlier thread's items is
  // the thread's first row, written only after the block scan), so no other
  // thread reads its end any more and a 4-byte result can take its place.  An
  // 8-byte result written there would cover two row ends, one of them
  // possibly another thread's current row: wider values get their own array.
  __shared__ T s_res_wide[sizeof(T) > 4 ? PADT : 1];
  T* s_res = sizeof(T) > 4 ? s_res_wide : reinterpret_cast<T*>(s_rend);
  __shared__ T s_wval[WARPS];
  __shared__ int32_t s_wrow[WARPS];
  __shared__ T s_prev_val[THREADS];
  __shared__ int32_t s_prev_row[THREADS];

  const int tid = threadIdx.x;
  const int64_t t = blockIdx.x;
  const int32_t r0 = tile_row[t], r1 = tile_row[t + 1];
  const int32_t e0 = tile_edge[t], e1 = tile_edge[t + 1];
  // A valid CSR gives nr + ne = TILE (the last tile less) with both >= 0.
  // Offsets that do not rise monotonically can give any split; clamping keeps
  // every shared-memory index inside the tile (the results are then
  // meaningless, but no access leaves its array).
  const int nr = min(max(r1 - r0, 0), TILE);
  const int ne = min(max(e1 - e0, 0), TILE - nr);

  if constexpr (VIRT) {  // row ends first: each edge finds its row among them
    for (int i = tid; i < nr; i += THREADS)
      s_rend[pad32(i)] = (int32_t)((int64_t)row_end[r0 + i] - e0);
    __syncthreads();
  }
  // 1. edges: stream col (or read the sources through the list), gather x
  {
    int32_t c[IPT];
    if constexpr (VIRT) {
      const int64_t start0 = r0 > 0 ? (int64_t)row_end[r0 - 1] : 0;  // row r0's first edge
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        const int j = u * THREADS + tid;
        c[u] = -1;
        if (j < ne) {
          int lo = 0, hi = nr;  // rows of the tile ending at or before edge j
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_rend[pad32(mid)] <= j) lo = mid + 1; else hi = mid;
          }
          const int64_t start = lo == 0 ? start0 : (int64_t)e0 + s_rend[pad32(lo - 1)];
          c[u] = __ldg(vadj + __ldg(voff + __ldg(vlist + r0 + lo)) + ((int64_t)e0 + j - start));
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        const int j = u * THREADS + tid;
        c[u] = j < ne ? __ldcs(col + e0 + j) : -1;
      }
    }
    T v[IPT];
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int32_t cu = c[u];
      bool ok = cu >= 0 && cu < nx;
      if constexpr (MASKED) ok = ok && ((__ldg(xmask + (cu >> 5)) >> (cu & 31)) & 1u);
      v[u] = ok ? ld_gather(x + (PROBE ? 0 : cu)) : Op::identity();
    }
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int j = u * THREADS + tid;
      if (j < ne) s_val[pad32(j)] = v[u];
    }
  }
  // 2. row ends relative to e0 (in [0, ne] for the tile's rows)
  if constexpr (!VIRT)
    for (int i = tid; i < nr; i += THREADS)
      s_rend[pad32(i)] = (int32_t)((int64_t)row_end[r0 + i] - e0);
  __syncthreads();

  // 3. sequential walk over this thread's merged items
  const int items = nr + ne;
  const int d0 = tid * IPT < items ? tid * IPT : items;
  const int d1 = d0 + IPT < items ? d0 + IPT : items;
  int i = (int)merge_path_search<true, int32_t>(d0, s_rend, nr, ne, 0);
  int j = d0 - i;
  __syncthreads();  // every search is done before row results replace row ends
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
        s_res[pad32(i)] = acc;
      }
      acc = Op::identity();
      ++i;
    } else {
      acc = Op::op(acc, s_val[pad32(j)]);
      ++j;
    }
  }
  // carry of this thread: (open row i, acc)

  // 4. block segmented inclusive scan of (row, value) over threads
  const int lane = tid & 31, w = tid >> 5;
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
    s_res[pad32(first_row)] = v;
  }
  __syncthreads();

  // 5. coalesced row results; tile carry for the row open at the tile end
  for (int r = tid; r < nr; r += THREADS) out[r0 + r] = s_res[pad32(r)];
  if (tid == THREADS - 1) {
    carry[t] = cval;     // the last thread's inclusive value is the open row's tile part
    carry_row[t] = r0 + crow;
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

// Tiling of one gather: per-tile start row / edge and the carry buffers.
struct TilePlan {
  int64_t nrows = 0, nedges = 0, ntiles = 0, tile = 0;
  int32_t* tile_row = nullptr;   // [ntiles+1]
  int32_t* tile_edge = nullptr;  // [ntiles+1]
  void* carry = nullptr;         // [ntiles] of 4-byte values
  int32_t* carry_row = nullptr;  // [ntiles]
};

constexpr int kTileThreads = 256;
constexpr int kTileIPT = 8;
constexpr int kTileItems = kTileThreads * kTileIPT;

// Allocate and fill a plan (cudaMalloc: the plan lives with its handle).
// carry_bytes: size of the gathered values (4, or 8 for SumF64).
template <typename RowEndT>
int plan_tiles(const RowEndT* row_end, int64_t nrows, int64_t nedges, TilePlan* p,
                cudaStream_t s, int carry_bytes = 4) {
  p->nrows = nrows;
  p->nedges = nedges;
  p->tile = kTileItems;
  p->ntiles = ceil_div(nrows + nedges, kTileItems);
  const size_t nb = sizeof(int32_t) * (size_t)(p->ntiles + 1);
  CG_CUDA(cudaMalloc((void**)&p->tile_row, nb));
  CG_CUDA(cudaMalloc((void**)&p->tile_edge, nb));
  CG_CUDA(cudaMalloc(&p->carry, (size_t)carry_bytes * (size_t)(p->ntiles + 1)));
  CG_CUDA(cudaMalloc((void**)&p->carry_row, nb));
  tile_partition_kernel<RowEndT><<<grid_for(p->ntiles + 1, 256), 256, 0, s>>>(
      row_end, nrows, nedges, kTileItems, p->ntiles, p->tile_row, p->tile_edge);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

inline void free_tile_plan(TilePlan* p) {
  cudaFree(p->tile_row);
  cudaFree(p->tile_edge);
  cudaFree(p->carry);
  cudaFree(p->carry_row);
  *p = TilePlan();
}

inline int64_t tile_plan_bytes(const TilePlan& p) { return 16 * (p.ntiles + 1); }

// Launch gather + fix-up.  row_end points at the first row's end.  xmask
// (optional): one bit per source, x read only where it is set.
template <class Op, bool PROBE, typename RowEndT>
int run_tile_gather(const TilePlan& p, const RowEndT* row_end, const int32_t* col,
                    const typename Op::T* x, int32_t nx, typename Op::T* out, cudaStream_t s,
                    const uint32_t* xmask = nullptr) {
  if (p.ntiles == 0) return CG_OK;
  if (xmask)
    gather_tile_kernel<Op, kTileThreads, kTileIPT, PROBE, RowEndT, true>
        <<<(unsigned)p.ntiles, kTileThreads, 0, s>>>(
            row_end, col, x, nx, p.tile_row, p.tile_edge, out,
            reinterpret_cast<typename Op::T*>(p.carry), p.carry_row, xmask);
  else
    gather_tile_kernel<Op, kTileThreads, kTileIPT, PROBE, RowEndT>
        <<<(unsigned)p.ntiles, kTileThreads, 0, s>>>(
            row_end, col, x, nx, p.tile_row, p.tile_edge, out,
            reinterpret_cast<typename Op::T*>(p.carry), p.carry_row);
  CG_LAUNCH_CHECK();
  carry_fixup_kernel<Op><<<grid_for(p.ntiles, 256, 4), 256, 0, s>>>(
      reinterpret_cast<const typename Op::T*>(p.carry), p.carry_row, p.ntiles, p.nrows, out);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

}  // namespace cg
