// Betweenness centrality from a set of sources (the BC application of the
// paper's Table V, run from 12 sources), by Brandes' algorithm over
// frontiers: the activeness side of the EdgeMap / VertexSubset API of
// Section IV, on the clustered graph (Section V; for BC the paper credits its
// speed-up to the renumbering, the working set being too small for
// segmenting to pay).
//
// Forward phase, one BFS level at a time from the source (level 0, sigma 1):
//   push (small frontier: its out-edges, one thread per edge, found through a
//         prefix sum of the frontier's out-degrees): an unvisited w gets level
//         L+1 by compare-and-swap and joins the next frontier; every edge into
//         a level-(L+1) vertex adds sigma[u] to sigma[w] with an FP64 atomic;
//   pull (large frontier, bottom-up: the merge-path tile gather over the
//         in-rows of the unvisited vertices, read through their list, of
//         x = sigma on the frontier, 0 elsewhere): an unvisited v whose sum is
//         non-zero gets level L+1 and sigma = the sum.
// sigma counts shortest paths: integers, exact in FP64 in any order below
// 2^53, so levels and sigma do not depend on the direction or the order.
// Pull is taken when (frontier out-edges) * alpha > E.
//
// Backward phase, deepest level first: for every u at level L,
//   delta[u] = sigma[u] * sum over out-neighbours w at level L+1 of
//              (1 + delta[w]) / sigma[w]
// as a gather over the out-rows of level L's vertices taken in the order of
// the level's list (a "virtual" CSR of that level: the tile gather reads each
// edge through the list), with x = (1 + delta) / sigma on level L+1 and
// 0 on every other level (out-neighbours of a level-L vertex lie at levels
// <= L+1, and levels <= L are still 0), by the same tile gather; the level
// lists are first put in (level, vertex ID) order, so the summation order is
// fixed and the results deterministic.  bc[u] += delta[u] for u != source.
#include <algorithm>
#include <vector>

#include "gather.cuh"
#include "handles.cuh"

struct cg_bc {
  int device = 0;
  int32_t V = 0;
  int64_t E = 0;
  const int64_t* in_off = nullptr;   // caller-owned in-edge CSR (pull)
  const int32_t* in_src = nullptr;
  const int64_t* out_off = nullptr;  // caller-owned out-edge CSR (push, backward)
  const int32_t* out_dst = nullptr;
  int32_t* level = nullptr;    // [V] BFS level of the current source (-1: unreached)
  double* sigma = nullptr;     // [V] shortest-path counts
  double* delta = nullptr;     // [V] dependencies
  double* xval = nullptr;      // [V] gathered values (see above), 0 elsewhere
  double* acc = nullptr;       // [V] gathered sums
  uint32_t* xbits = nullptr;   // [V/32 + 1] one bit per vertex: xval may be non-zero
  int32_t* lists = nullptr;    // [V] reached vertices, level after level
  int32_t* deg = nullptr;      // [V] out-degrees of one level's vertices
  int64_t* rend = nullptr;     // [V+1] their exclusive prefix (rend[n] = total)
  int32_t* counter = nullptr;  // [1] next free position in lists
  int32_t* ids = nullptr;      // [V] sort scratch: reached vertices in ID order
  uint32_t* keys = nullptr;    // [V] sort scratch: their levels
  uint32_t* keys_out = nullptr;  // [V]
  int64_t* h_pin = nullptr;    // pinned host words for the per-level counts
  int32_t* vt_row = nullptr;   // tiles of a level's virtual CSR
  int32_t* vt_edge = nullptr;
  double* vt_carry = nullptr;
  int32_t* vt_carry_row = nullptr;
  int64_t vt_cap = 0;
  double alpha = 16.0;
  std::vector<int64_t> lbase;  // level bounds in `lists` of the last source
  int32_t last_source = -1;
  int32_t push_levels = 0, pull_levels = 0;
};

namespace cg {
namespace {

constexpr int kThreads = 256;

__global__ void bc_reset_kernel(int32_t V, int32_t* __restrict__ level,
                                double* __restrict__ sigma, double* __restrict__ delta,
                                double* __restrict__ xval, uint32_t* __restrict__ xbits) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    level[v] = -1;
    sigma[v] = 0.0;
    delta[v] = 0.0;
    xval[v] = 0.0;
    if ((v & 31) == 0) xbits[v >> 5] = 0u;
  }
}

__device__ __forceinline__ void set_bit(uint32_t* bits, int32_t v, bool on) {
  if (on)
    atomicOr(bits + (v >> 5), 1u << (v & 31));
  else
    atomicAnd(bits + (v >> 5), ~(1u << (v & 31)));
}

__global__ void bc_seed_kernel(int32_t s, int32_t* __restrict__ level, double* __restrict__ sigma,
                               double* __restrict__ xval, uint32_t* __restrict__ xbits,
                               int32_t* __restrict__ lists, int32_t* __restrict__ counter) {
  level[s] = 0;
  sigma[s] = 1.0;
  xval[s] = 1.0;
  set_bit(xbits, s, true);
  lists[0] = s;
  *counter = 1;
}

// Row lengths in a CSR (off: the out- or in-edge offsets) for the vertices of
// a list (taken from the expanded CSR's own offsets, so every expanded edge
// lies inside its row).
__global__ void list_degree_kernel(const int32_t* __restrict__ list, int64_t n,
                                   const int64_t* __restrict__ off, int32_t* __restrict__ deg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = list[i];
    deg[i] = (int32_t)(off[u + 1] - off[u]);
  }
}

// Append v to lists at a position from one atomic per warp.
__device__ __forceinline__ void append(bool take, int32_t v, int32_t* lists, int32_t* counter) {
  const unsigned m = __ballot_sync(0xffffffffu, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  int32_t base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
  if (take) lists[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// The out-edges [0, m) of a list's vertices laid end to end (row i = list
// position i, starting at rend[i]) are cut into merge-path tiles of rows +
// edges (tile_row / tile_edge, as for the gather); the block of tile t keeps
// the starts rend[r0 .. r1] of the tile's rows in shared memory, so each of
// its edges finds its row with a binary search in shared memory.  Returns
// the number of row starts loaded (0: the tile has no edges).
__device__ __forceinline__ int load_tile_rows(const int64_t* __restrict__ rend, int64_t n,
                                              const int32_t* __restrict__ tile_row,
                                              const int32_t* __restrict__ tile_edge,
                                              int64_t* s_start, int64_t& r0, int64_t& e0,
                                              int64_t& e1) {
  const int64_t t = blockIdx.x;
  r0 = tile_row[t];
  e0 = tile_edge[t];
  e1 = tile_edge[t + 1];
  if (e0 >= e1) return 0;
  const int64_t rl = tile_row[t + 1] < n - 1 ? tile_row[t + 1] : n - 1;
  const int cnt = (int)(rl - r0 + 1);  // <= kTileItems + 1
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) s_start[j] = rend[r0 + j];
  __syncthreads();
  return cnt;
}

// last j in [0, cnt) with s_start[j] <= k (s_start ascending, s_start[0] <= k)
__device__ __forceinline__ int tile_row_of(const int64_t* s_start, int cnt, int64_t k) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s_start[mid] <= k) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Push: the frontier's (list, n vertices) out-edges, a tile per block.
__global__ void __launch_bounds__(kThreads)
push_kernel(const int32_t* __restrict__ list, int64_t n, const int64_t* __restrict__ rend,
            const int32_t* __restrict__ tile_row, const int32_t* __restrict__ tile_edge,
            const int64_t* __restrict__ out_off, const int32_t* __restrict__ out_dst, int32_t L,
            int32_t* __restrict__ level, double* __restrict__ sigma,
            int32_t* __restrict__ lists, int32_t* __restrict__ counter) {
  __shared__ int64_t s_start[kTileItems + 1];
  int64_t r0, e0, e1;
  const int cnt = load_tile_rows(rend, n, tile_row, tile_edge, s_start, r0, e0, e1);
  if (cnt == 0) return;
  for (int64_t k0 = e0; k0 < e1; k0 += blockDim.x) {
    const int64_t k = k0 + threadIdx.x;  // the warp stays converged for the append
    bool take = false;
    int32_t w = 0;
    if (k < e1) {
      const int j = tile_row_of(s_start, cnt, k);
      const int32_t u = list[r0 + j];
      w = out_dst[out_off[u] + (k - s_start[j])];
      // a target seen visited on an earlier level needs no atomic; one that
      // reads unvisited takes the compare-and-swap (it may lose to another
      // edge of this level, which then reads L + 1)
      int32_t old = __ldcg(level + w);
      if (old == -1) old = atomicCAS(level + w, -1, L + 1);
      take = old == -1;
      if (old == -1 || old == L + 1) atomicAdd(sigma + w, sigma[u]);
    }
    append(take, w, lists, counter);
  }
}

// Bottom-up step: the unvisited vertices that have in-edges (their IDs in
// ascending order) ...
__global__ void unvisited_flag_kernel(int32_t V, const int32_t* __restrict__ level,
                                      const int64_t* __restrict__ in_off,
                                      int32_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = level[v] == -1 && in_off[v + 1] > in_off[v];
}

__global__ void unvisited_compact_kernel(int32_t V, const int32_t* __restrict__ level,
                                         const int64_t* __restrict__ in_off,
                                         const int64_t* __restrict__ pos,
                                         int32_t* __restrict__ ids) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x)
    if (level[v] == -1 && in_off[v + 1] > in_off[v]) ids[pos[v]] = (int32_t)v;
}

// ... and after the gather of their in-rows: one with a non-zero sum (a
// frontier in-neighbour) is on level L+1.
__global__ void pull_update_kernel(const int32_t* __restrict__ ids, int64_t n,
                                   const double* __restrict__ acc, int32_t L,
                                   int32_t* __restrict__ level, double* __restrict__ sigma,
                                   int32_t* __restrict__ lists, int32_t* __restrict__ counter) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;  // the warp stays converged for the append
    bool take = false;
    int32_t v = 0;
    if (i < n) {
      v = ids[i];
      const double a = acc[i];
      if (a != 0.0) {
        level[v] = L + 1;
        sigma[v] = a;
        take = true;
      }
    }
    append(take, v, lists, counter);
  }
}

// x over the vertices of a list: sigma (forward frontier) or 0, with the
// vertices' bits in xbits.
__global__ void set_x_kernel(const int32_t* __restrict__ list, int64_t n,
                             const double* __restrict__ sigma, double* __restrict__ xval,
                             uint32_t* __restrict__ xbits, bool clear) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = list[i];
    xval[u] = clear ? 0.0 : sigma[u];
    set_bit(xbits, u, !clear);
  }
}

// The deepest level: delta = 0, x = 1 / sigma.
__global__ void deepest_kernel(const int32_t* __restrict__ list, int64_t n,
                               const double* __restrict__ sigma, double* __restrict__ xval,
                               uint32_t* __restrict__ xbits) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = list[i];
    xval[u] = 1.0 / sigma[u];
    set_bit(xbits, u, true);
  }
}

// delta of level L from the gathered sums; bc += delta (not for the source);
// x = (1 + delta) / sigma for the next level up.
__global__ void dependency_kernel(const int32_t* __restrict__ list, int64_t n,
                                  const double* __restrict__ sums, const double* __restrict__ sigma,
                                  double* __restrict__ delta, double* __restrict__ xval,
                                  uint32_t* __restrict__ xbits, double* __restrict__ bc,
                                  int32_t source) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = list[i];
    const double d = sigma[u] * sums[i];
    delta[u] = d;
    xval[u] = (1.0 + d) / sigma[u];
    set_bit(xbits, u, true);
    if (u != source) bc[u] += d;
  }
}

// Reached vertices in ascending ID order (pos: exclusive prefix of reached).
__global__ void reached_flag_kernel(int32_t V, const int32_t* __restrict__ level,
                                    int32_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = level[v] >= 0;
}

__global__ void compact_kernel(int32_t V, const int32_t* __restrict__ level,
                               const int64_t* __restrict__ pos, int32_t* __restrict__ ids,
                               uint32_t* __restrict__ keys) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = level[v];
    if (l >= 0) {
      ids[pos[v]] = (int32_t)v;
      keys[pos[v]] = (uint32_t)l;
    }
  }
}

__global__ void row_of_edge_kernel(const int64_t* __restrict__ off, int32_t V,
                                   int32_t* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nw)
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) dst[e] = (int32_t)v;
}

int read_i64(cg_bc* h, const int64_t* dev, int64_t* out, cudaStream_t s) {
  CG_CUDA(cudaMemcpyAsync(h->h_pin, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  *out = h->h_pin[0];
  return CG_OK;
}

int read_i32(cg_bc* h, const int32_t* dev, int32_t* out, cudaStream_t s) {
  CG_CUDA(cudaMemcpyAsync(h->h_pin, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  *out = *reinterpret_cast<int32_t*>(h->h_pin);
  return CG_OK;
}

// Degrees of list[0, n) and their prefix; *m = total out-edges.
int level_rows(cg_bc* h, const int32_t* list, int64_t n, int64_t* m, cudaStream_t s) {
  list_degree_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(list, n, h->out_off, h->deg);
  CG_LAUNCH_CHECK();
  CG_TRY(exclusive_scan_i32_to_i64(h->deg, h->rend, n, s));
  return read_i64(h, h->rend + n, m, s);
}

int grow_vt(cg_bc* h, int64_t ntiles);

// Merge-path tiles of a list's n rows and m out-edges (rend: row starts,
// rend[n] = m) into h->vt_row / h->vt_edge; *ntiles = their number.
int level_tiles(cg_bc* h, int64_t n, int64_t m, int64_t* ntiles, cudaStream_t s) {
  *ntiles = ceil_div(n + m, kTileItems);
  CG_TRY(grow_vt(h, *ntiles));
  tile_partition_kernel<int64_t><<<grid_for(*ntiles + 1, 256), 256, 0, s>>>(
      h->rend + 1, n, m, kTileItems, *ntiles, h->vt_row, h->vt_edge);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int grow_vt(cg_bc* h, int64_t ntiles) {
  if (ntiles + 1 <= h->vt_cap) return CG_OK;
  cudaFree(h->vt_row);
  cudaFree(h->vt_edge);
  cudaFree(h->vt_carry);
  cudaFree(h->vt_carry_row);
  h->vt_row = h->vt_edge = h->vt_carry_row = nullptr;
  h->vt_carry = nullptr;
  h->vt_cap = 0;
  const size_t c = (size_t)(ntiles + 1);
  CG_CUDA(cudaMalloc((void**)&h->vt_row, 4 * c));
  CG_CUDA(cudaMalloc((void**)&h->vt_edge, 4 * c));
  CG_CUDA(cudaMalloc((void**)&h->vt_carry, 8 * c));
  CG_CUDA(cudaMalloc((void**)&h->vt_carry_row, 4 * c));
  h->vt_cap = ntiles + 1;
  return CG_OK;
}

// Lay the level lists out in (level, vertex ID) order: the appends of the
// forward phase come in whatever order the atomics give, and the backward
// sums are associated by position in these lists.  A compaction of the
// reached vertices in ID order, then a stable radix sort on the level.
int order_levels(cg_bc* h, int32_t depth, cudaStream_t s) {
  const int32_t V = h->V;
  const int64_t n = h->lbase[depth];
  reached_flag_kernel<<<grid_for(V, kThreads), kThreads, 0, s>>>(V, h->level, h->deg);
  CG_LAUNCH_CHECK();
  CG_TRY(exclusive_scan_i32_to_i64(h->deg, h->rend, V, s));
  compact_kernel<<<grid_for(V, kThreads), kThreads, 0, s>>>(V, h->level, h->rend, h->ids,
                                                            h->keys);
  CG_LAUNCH_CHECK();
  int bits = 1;
  while (bits < 32 && (int64_t(1) << bits) < (int64_t)depth) ++bits;
  return radix_sort_pairs(h->keys, h->ids, h->keys_out, h->lists, n, bits, s);
}

// One bottom-up level: the unvisited vertices that have in-edges (ids, in
// ID order) gather x = sigma on the frontier (0 elsewhere, tested through
// xbits) over their in-rows laid end to end; a non-zero sum puts a vertex on
// level L+1 with that sum as its path count.  Visited vertices' rows are
// never read.
int pull_level(cg_bc* h, int32_t L, cudaStream_t s) {
  const int32_t V = h->V;
  unvisited_flag_kernel<<<grid_for(V, kThreads), kThreads, 0, s>>>(V, h->level, h->in_off,
                                                                    h->deg);
  CG_LAUNCH_CHECK();
  CG_TRY(exclusive_scan_i32_to_i64(h->deg, h->rend, V, s));
  unvisited_compact_kernel<<<grid_for(V, kThreads), kThreads, 0, s>>>(V, h->level, h->in_off,
                                                                       h->rend, h->ids);
  CG_LAUNCH_CHECK();
  int64_t n = 0, m = 0;
  CG_TRY(read_i64(h, h->rend + V, &n, s));
  if (n == 0) return CG_OK;
  list_degree_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(h->ids, n, h->in_off, h->deg);
  CG_LAUNCH_CHECK();
  CG_TRY(exclusive_scan_i32_to_i64(h->deg, h->rend, n, s));
  CG_TRY(read_i64(h, h->rend + n, &m, s));
  if (m == 0) return CG_OK;
  int64_t ntiles = 0;
  CG_TRY(level_tiles(h, n, m, &ntiles, s));
  // the in-rows of the listed vertices, read through the list (no copy)
  gather_tile_kernel<SumF64, kTileThreads, kTileIPT, false, int64_t, true, true>
      <<<(unsigned)ntiles, kTileThreads, 0, s>>>(h->rend + 1, nullptr, h->xval, V, h->vt_row,
                                                 h->vt_edge, h->acc, h->vt_carry,
                                                 h->vt_carry_row, h->xbits, h->ids, h->in_off,
                                                 h->in_src);
  CG_LAUNCH_CHECK();
  carry_fixup_kernel<SumF64><<<grid_for(ntiles, 256, 4), 256, 0, s>>>(h->vt_carry,
                                                                     h->vt_carry_row, ntiles, n,
                                                                     h->acc);
  CG_LAUNCH_CHECK();
  pull_update_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(h->ids, n, h->acc, L, h->level,
                                                                h->sigma, h->lists, h->counter);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int run_source(cg_bc* h, int32_t src, double* bc, cudaStream_t s) {
  const int32_t V = h->V;
  bc_reset_kernel<<<grid_for(V, kThreads), kThreads, 0, s>>>(V, h->level, h->sigma, h->delta,
                                                               h->xval, h->xbits);
  CG_LAUNCH_CHECK();
  bc_seed_kernel<<<1, 1, 0, s>>>(src, h->level, h->sigma, h->xval, h->xbits, h->lists,
                                 h->counter);
  CG_LAUNCH_CHECK();
  h->lbase.assign(1, 0);
  h->lbase.push_back(1);
  h->push_levels = h->pull_levels = 0;
  // forward: one level per round until a level adds nobody
  for (int32_t L = 0;; ++L) {
    const int64_t b0 = h->lbase[L], n = h->lbase[L + 1] - b0;
    const int32_t* list = h->lists + b0;
    int64_t m = 0;
    CG_TRY(level_rows(h, list, n, &m, s));
    if (m > 0) {
      if ((double)m * h->alpha > (double)h->E) {  // pull (bottom-up)
        CG_TRY(pull_level(h, L, s));
        ++h->pull_levels;
      } else {  // push from the frontier's out-edges
        int64_t ntiles = 0;
        CG_TRY(level_tiles(h, n, m, &ntiles, s));
        push_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(list, n, h->rend, h->vt_row,
                                                          h->vt_edge, h->out_off, h->out_dst, L,
                                                          h->level, h->sigma, h->lists,
                                                          h->counter);
        CG_LAUNCH_CHECK();
        ++h->push_levels;
      }
    }
    int32_t cnt = 0;
    CG_TRY(read_i32(h, h->counter, &cnt, s));
    if (cnt == h->lbase[L + 1]) break;  // nothing new: L is the deepest level
    h->lbase.push_back(cnt);
    // the frontier moves on: x = sigma on level L+1 only
    set_x_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(list, n, h->sigma, h->xval, h->xbits,
                                                            true);
    CG_LAUNCH_CHECK();
    const int64_t n1 = cnt - h->lbase[L + 1];
    set_x_kernel<<<grid_for(n1, kThreads), kThreads, 0, s>>>(h->lists + h->lbase[L + 1], n1,
                                                             h->sigma, h->xval, h->xbits, false);
    CG_LAUNCH_CHECK();
  }
  const int32_t depth = (int32_t)h->lbase.size() - 1;  // levels 0 .. depth-1
  CG_TRY(order_levels(h, depth, s));
  {
    const int64_t b = h->lbase[depth - 1], n = h->lbase[depth] - b;
    deepest_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(h->lists + b, n, h->sigma,
                                                              h->xval, h->xbits);
    CG_LAUNCH_CHECK();
  }
  // backward: levels depth-2 .. 0
  for (int32_t L = depth - 2; L >= 0; --L) {
    const int64_t b0 = h->lbase[L], n = h->lbase[L + 1] - b0;
    const int32_t* list = h->lists + b0;
    int64_t m = 0;
    CG_TRY(level_rows(h, list, n, &m, s));
    if (m > 0) {
      int64_t ntiles = 0;
      CG_TRY(level_tiles(h, n, m, &ntiles, s));
      // the out-rows of level L's vertices, read through the level list
      gather_tile_kernel<SumF64, kTileThreads, kTileIPT, false, int64_t, true, true>
          <<<(unsigned)ntiles, kTileThreads, 0, s>>>(h->rend + 1, nullptr, h->xval, V,
                                                     h->vt_row, h->vt_edge, h->acc, h->vt_carry,
                                                     h->vt_carry_row, h->xbits, list, h->out_off,
                                                     h->out_dst);
      CG_LAUNCH_CHECK();
      carry_fixup_kernel<SumF64><<<grid_for(ntiles, 256, 4), 256, 0, s>>>(
          h->vt_carry, h->vt_carry_row, ntiles, n, h->acc);
      CG_LAUNCH_CHECK();
    } else {
      CG_CUDA(cudaMemsetAsync(h->acc, 0, sizeof(double) * (size_t)n, s));
    }
    dependency_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(list, n, h->acc, h->sigma,
                                                                h->delta, h->xval, h->xbits, bc,
                                                                src);
    CG_LAUNCH_CHECK();
  }
  h->last_source = src;
  return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int cg_transpose_csr(const int64_t* in_offsets, const int32_t* in_src, int32_t V, int64_t E,
                     int64_t* out_offsets, int32_t* out_dst, cudaStream_t stream) {
  CG_ARG(V >= 1 && E >= 0 && E < 0x7FFFFFFFLL, "cg_transpose_csr: V >= 1 and 0 <= E < 2^31-1");
  CG_ARG(in_offsets && out_offsets && (E == 0 || (in_src && out_dst)),
         "cg_transpose_csr: null pointer argument");
  CG_TRY(validate_csr(in_offsets, in_src, V, E, stream));
  int32_t* deg = nullptr;
  int32_t* rows = nullptr;
  uint32_t* kout = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&deg, sizeof(int32_t) * (size_t)V, stream);
  int st = e == cudaSuccess ? CG_OK : cuda_fail(e, "cg_transpose_csr", __FILE__, __LINE__);
  if (st == CG_OK) st = cg_out_degree(in_src, E, V, deg, stream);
  if (st == CG_OK) st = exclusive_scan_i32_to_i64(deg, out_offsets, V, stream);
  if (st == CG_OK && E > 0) {
    e = cudaMallocAsync((void**)&rows, sizeof(int32_t) * (size_t)E, stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&kout, sizeof(uint32_t) * (size_t)E, stream);
    if (e == cudaSuccess) {
      row_of_edge_kernel<<<grid_for((int64_t)V * 32, 256), 256, 0, stream>>>(in_offsets, V, rows);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_fail(e, "cg_transpose_csr", __FILE__, __LINE__);
    int bits = 1;
    while (bits < 32 && (int64_t(1) << bits) < (int64_t)V) ++bits;
    // stable sort of the edges by source keeps each out-row in ascending
    // destination order (the in-edge CSR lists its rows in that order)
    if (st == CG_OK)
      st = radix_sort_pairs(reinterpret_cast<const uint32_t*>(in_src), rows, kout, out_dst, E,
                            bits, stream);
  }
  if (deg) cudaFreeAsync(deg, stream);
  if (rows) cudaFreeAsync(rows, stream);
  if (kout) cudaFreeAsync(kout, stream);
  return st;
}

int bc_create(const int64_t* in_offsets, const int32_t* in_src, const int64_t* out_offsets,
              const int32_t* out_dst, int32_t V, int64_t E, cg_bc** out, cudaStream_t stream) {
  CG_ARG(out != nullptr, "bc_create: out is NULL");
  *out = nullptr;
  CG_ARG(V >= 1 && E >= 0 && E < 0x7FFFFFFFLL, "bc_create: V >= 1 and 0 <= E < 2^31-1");
  CG_ARG(in_offsets && out_offsets && (E == 0 || (in_src && out_dst)),
         "bc_create: null pointer argument");
  CG_TRY(validate_csr(in_offsets, in_src, V, E, stream));
  CG_TRY(validate_csr(out_offsets, out_dst, V, E, stream));
  cg_bc* h = new cg_bc();
  cudaGetDevice(&h->device);
  h->V = V;
  h->E = E;
  h->in_off = in_offsets;
  h->in_src = in_src;
  h->out_off = out_offsets;
  h->out_dst = out_dst;
  const size_t v4 = sizeof(int32_t) * (size_t)V, v8 = sizeof(double) * (size_t)V;
  cudaError_t e = cudaMalloc((void**)&h->level, v4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->sigma, v8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->delta, v8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->xval, v8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->acc, v8);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&h->xbits, sizeof(uint32_t) * ((size_t)V / 32 + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->lists, v4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->deg, v4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->rend, sizeof(int64_t) * ((size_t)V + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->counter, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->ids, v4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->keys, v4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->keys_out, v4);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&h->h_pin, 2 * sizeof(int64_t), 0);
  int st = e == cudaSuccess ? CG_OK : cuda_fail(e, "bc_create", __FILE__, __LINE__);
  if (st == CG_OK) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = cuda_fail(e, "bc_create", __FILE__, __LINE__);
  }
  if (st != CG_OK) {
    bc_destroy(h);
    return st;
  }
  *out = h;
  return CG_OK;
}

int bc_destroy(cg_bc* h) {
  if (!h) return CG_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->level);
  cudaFree(h->sigma);
  cudaFree(h->delta);
  cudaFree(h->xval);
  cudaFree(h->acc);
  cudaFree(h->xbits);
  cudaFree(h->lists);
  cudaFree(h->deg);
  cudaFree(h->rend);
  cudaFree(h->counter);
  cudaFree(h->ids);
  cudaFree(h->keys);
  cudaFree(h->keys_out);
  cudaFree(h->vt_row);
  cudaFree(h->vt_edge);
  cudaFree(h->vt_carry);
  cudaFree(h->vt_carry_row);
  if (h->h_pin) cudaFreeHost(h->h_pin);
  if (cur != h->device) cudaSetDevice(cur);
  delete h;
  return CG_OK;
}

int bc_set_direction(cg_bc* h, double alpha) {
  CG_ARG(h != nullptr, "bc_set_direction: null handle");
  CG_ARG(alpha >= 0.0, "bc_set_direction: alpha must be >= 0");
  h->alpha = alpha;
  return CG_OK;
}

int bc_run(cg_bc* h, const int32_t* sources, int32_t nsources, double* bc, cudaStream_t stream) {
  CG_ARG(h != nullptr, "bc_run: null handle");
  CG_ARG(nsources >= 0 && (nsources == 0 || sources) && bc, "bc_run: bad arguments");
  for (int32_t i = 0; i < nsources; ++i)
    CG_ARG(sources[i] >= 0 && sources[i] < h->V, "bc_run: source %d outside [0, %d)",
           sources[i], h->V);
  for (int32_t i = 0; i < nsources; ++i) CG_TRY(run_source(h, sources[i], bc, stream));
  return CG_OK;
}

int bc_source_state(const cg_bc* h, int32_t* level, double* sigma, double* delta,
                    int32_t* depth, int32_t* push_levels, int32_t* pull_levels,
                    cudaStream_t stream) {
  CG_ARG(h != nullptr, "bc_source_state: null handle");
  CG_ARG(h->last_source >= 0, "bc_source_state: no source has run yet");
  const size_t v4 = sizeof(int32_t) * (size_t)h->V, v8 = sizeof(double) * (size_t)h->V;
  if (level) CG_CUDA(cudaMemcpyAsync(level, h->level, v4, cudaMemcpyDeviceToDevice, stream));
  if (sigma) CG_CUDA(cudaMemcpyAsync(sigma, h->sigma, v8, cudaMemcpyDeviceToDevice, stream));
  if (delta) CG_CUDA(cudaMemcpyAsync(delta, h->delta, v8, cudaMemcpyDeviceToDevice, stream));
  if (depth) *depth = (int32_t)h->lbase.size() - 1;
  if (push_levels) *push_levels = h->push_levels;
  if (pull_levels) *pull_levels = h->pull_levels;
  return CG_OK;
}

}  // extern "C"
