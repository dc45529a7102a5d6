// CSR segmenting preprocessing (Algorithm 2, Section III-A) on the GPU.
//
// Steps (all device work except reading a few sizes back):
//   A. per destination row: how many segments its in-edges come from;
//   B. per (row, segment) pair: the edge count, rows in order, segments
//      ascending inside a row;
//   C. a stable sort of the pairs by segment gives the segment-major row
//      order (segment by segment, destinations ascending inside each) =
//      the subgraphs' rows, idxMap and row lengths;
//   D. every edge is placed in its subgraph row, keeping parent order;
//   E. merge-block indices (blockStarts / blockEnds of Algorithm 4);
//   F. the gather tiling and the intermBuf of the handle.
#include <algorithm>
#include <vector>

#include "handles.cuh"

namespace cg {
namespace {

constexpr int kBuildWarps = 4;
constexpr int kBuildThreads = kBuildWarps * 32;
constexpr int kMaxSegments = 1024;

// Segment of source u: last s with bounds[s] <= u (empty segments skipped).
__device__ __forceinline__ int seg_of(int32_t u, const int32_t* sb, int k) {
  int lo = 0, hi = k + 1;  // upper_bound over sb[0..k]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (sb[mid] <= u) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

__global__ void validate_csr_kernel(const int64_t* __restrict__ offsets,
                                    const int32_t* __restrict__ src, int32_t V, int64_t E,
                                    unsigned long long* __restrict__ bad) {
  unsigned long long nbad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t v = t0; v < V; v += stride) nbad += offsets[v + 1] < offsets[v];
  if (t0 == 0) nbad += (offsets[0] != 0) + (offsets[V] != E);
  for (int64_t e = t0; e < E; e += stride) {
    const int32_t u = __ldcs(src + e);
    nbad += (u < 0 || u >= V);
  }
  nbad = warp_sum(nbad);
  if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, nbad);
}

// A. number of distinct segments among each row's sources.
__global__ void row_nseg_kernel(const int64_t* __restrict__ offsets,
                                const int32_t* __restrict__ src, int32_t V,
                                const int32_t* __restrict__ bounds, int k,
                                int32_t* __restrict__ nseg) {
  extern __shared__ int32_t sm[];
  int32_t* sb = sm;                                   // [k+1]
  const int words = (k + 31) >> 5;
  uint32_t* bm = reinterpret_cast<uint32_t*>(sb + ((k + 1 + 3) & ~3));  // [warps][words]
  for (int i = threadIdx.x; i <= k; i += blockDim.x) sb[i] = bounds[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* mybm = bm + w * words;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nwarps) {
    for (int q = lane; q < words; q += 32) mybm[q] = 0u;
    __syncwarp();
    const int64_t lo = offsets[v], hi = offsets[v + 1];
    for (int64_t e = lo + lane; e < hi; e += 32) {
      const int s = seg_of(src[e], sb, k);
      atomicOr(mybm + (s >> 5), 1u << (s & 31));
    }
    __syncwarp();
    int c = 0;
    for (int q = lane; q < words; q += 32) c += __popc(mybm[q]);
    c = warp_sum(c);
    if (lane == 0) nseg[v] = c;
    __syncwarp();
  }
}

// B. (segment, row, count) for every (row, segment) pair; a row's pairs are
// written at pos[v] in ascending segment order.
__global__ void row_pairs_kernel(const int64_t* __restrict__ offsets,
                                 const int32_t* __restrict__ src, int32_t V,
                                 const int32_t* __restrict__ bounds, int k,
                                 const int64_t* __restrict__ pos, uint32_t* __restrict__ pseg,
                                 int32_t* __restrict__ prow, int32_t* __restrict__ pcnt) {
  extern __shared__ int32_t sm[];
  const int words = (k + 31) >> 5;
  int32_t* sb = sm;                                             // [k+1]
  int32_t* cnt = sb + ((k + 1 + 3) & ~3);                       // [warps][k]
  uint32_t* bm = reinterpret_cast<uint32_t*>(cnt + kBuildWarps * k);  // [warps][words]
  for (int i = threadIdx.x; i <= k; i += blockDim.x) sb[i] = bounds[i];
  for (int i = threadIdx.x; i < kBuildWarps * k; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t* mycnt = cnt + w * k;
  uint32_t* mybm = bm + w * words;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nwarps) {
    for (int q = lane; q < words; q += 32) mybm[q] = 0u;
    __syncwarp();
    const int64_t lo = offsets[v], hi = offsets[v + 1];
    for (int64_t e = lo + lane; e < hi; e += 32) {
      const int s = seg_of(src[e], sb, k);
      atomicOr(mybm + (s >> 5), 1u << (s & 31));
      atomicAdd(mycnt + s, 1);
    }
    __syncwarp();
    // enumerate set bits word by word; lane q owns words q, q+32, ... (k <= 1024: one word)
    int64_t base = pos[v];
    for (int q0 = 0; q0 < words; q0 += 32) {
      const int q = q0 + lane;
      uint32_t word = q < words ? mybm[q] : 0u;
      const int n = __popc(word);
      int incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int64_t p = base + incl - n;
      while (word) {
        const int b = __ffs(word) - 1;
        const int s = q * 32 + b;
        pseg[p] = (uint32_t)s;
        prow[p] = (int32_t)v;
        pcnt[p] = mycnt[s];
        mycnt[s] = 0;
        ++p;
        word &= word - 1u;
      }
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
  }
}

__global__ void iota_kernel(int32_t* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// C. segment-major rows from the sorted pair order.
__global__ void pairs_to_rows_kernel(const int32_t* __restrict__ perm,
                                     const int32_t* __restrict__ prow,
                                     const int32_t* __restrict__ pcnt, int64_t n,
                                     int32_t* __restrict__ idx_map, int32_t* __restrict__ rowlen,
                                     int32_t* __restrict__ inv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[i];
    idx_map[i] = prow[p];
    rowlen[i] = pcnt[p];
    inv[p] = (int32_t)i;
  }
}

// row_base[s] = first sorted pair with segment >= s (k+1 threads).
__global__ void segment_starts_kernel(const uint32_t* __restrict__ skey, int64_t n, int k,
                                      int64_t* __restrict__ row_base) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > k) return;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)skey[mid] < s) lo = mid + 1; else hi = mid;
  }
  row_base[s] = lo;
}

__global__ void to_i32_kernel(const int64_t* __restrict__ in, int64_t n,
                              int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

// D. place every edge: cur[s] = next free slot of this row's segment-s subrow.
__global__ void scatter_edges_kernel(const int64_t* __restrict__ offsets,
                                     const int32_t* __restrict__ src, int32_t V,
                                     const int32_t* __restrict__ bounds, int k,
                                     const int64_t* __restrict__ pos,
                                     const uint32_t* __restrict__ pseg,
                                     const int32_t* __restrict__ inv,
                                     const int64_t* __restrict__ rp, int32_t* __restrict__ col) {
  extern __shared__ int64_t sm64[];
  int64_t* cur = sm64;                                          // [warps][k]
  int32_t* sb = reinterpret_cast<int32_t*>(cur + kBuildWarps * k);  // [k+1]
  for (int i = threadIdx.x; i <= k; i += blockDim.x) sb[i] = bounds[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int64_t* mycur = cur + w * k;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nwarps) {
    for (int64_t p = pos[v] + lane; p < pos[v + 1]; p += 32) mycur[pseg[p]] = rp[inv[p]];
    __syncwarp();
    const int64_t lo = offsets[v], hi = offsets[v + 1];
    for (int64_t e0 = lo; e0 < hi; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool ok = e < hi;
      const int32_t u = ok ? src[e] : 0;
      const int s = ok ? seg_of(u, sb, k) : 0;
      const unsigned key = ok ? (unsigned)s : (0x10000u | (unsigned)lane);
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (ok) col[mycur[s] + __popc(peers & lt)] = u;
      __syncwarp();
      if (ok && lane == __ffs(peers) - 1) mycur[s] += __popc(peers);
      __syncwarp();
    }
  }
}

// E. merge-block indices.
__global__ void blk_prefill_kernel(const int64_t* __restrict__ row_base, int k, int nb,
                                   int32_t* __restrict__ blk) {
  const int64_t n = (int64_t)k * (nb + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    blk[i] = (int32_t)row_base[i / (nb + 1)];
}

__global__ void blk_rows_kernel(const int64_t* __restrict__ row_base, int k,
                                const int32_t* __restrict__ idx_map, int64_t rows, int B, int nb,
                                int32_t* __restrict__ blk) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = k + 1;  // segment of row i: last s with row_base[s] <= i
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (row_base[mid] <= i) lo = mid + 1; else hi = mid;
    }
    const int s = lo - 1;
    int32_t* b_s = blk + (int64_t)s * (nb + 1);
    const int bk = idx_map[i] / B;
    const int pbk = (i == row_base[s]) ? -1 : idx_map[i - 1] / B;
    for (int b = pbk + 1; b <= bk; ++b) b_s[b] = (int32_t)i;
    if (i == row_base[s + 1] - 1)
      for (int b = bk + 1; b <= nb; ++b) b_s[b] = (int32_t)row_base[s + 1];
  }
}

// Export helpers.
__global__ void to_i64_kernel(const int32_t* __restrict__ in, int64_t n,
                              int64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// Block-major merge index (blk[b*k + s]) -> segment-major local rows
// (out[s*(nb+1) + b] = blk[b*k + s] - row_base[s]), the oracle's layout.
__global__ void blk_local_kernel(const int32_t* __restrict__ blk, const int64_t* __restrict__ rb,
                                 int k, int nb, int32_t* __restrict__ out) {
  const int64_t n = (int64_t)k * (nb + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = i / (nb + 1), b = i % (nb + 1);
    out[i] = (int32_t)(blk[b * k + sg] - rb[sg]);
  }
}

// Segment-major (blk_sm[s*(nb+1) + b]) -> block-major (blk[b*k + s]): a merge
// block's first rows of all segments are then one contiguous run.
__global__ void blk_transpose_kernel(const int32_t* __restrict__ blk_sm, int k, int nb,
                                     int32_t* __restrict__ blk) {
  const int64_t n = (int64_t)k * (nb + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / k, sg = i % k;
    blk[i] = blk_sm[sg * (nb + 1) + b];
  }
}

struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <typename T>
  cudaError_t get(T** p, size_t n) {
    cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (n > 0 ? n : 1), s);
    if (e == cudaSuccess) ptrs.push_back((void*)*p);
    return e;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

int build_impl(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E, int32_t k,
               const std::vector<int64_t>& bounds, int32_t B, cg_segmented* g, cudaStream_t s) {
  Scratch tmp(s);
  int32_t* d_bounds = nullptr;
  CG_CUDA(tmp.get(&d_bounds, k + 1));
  {
    std::vector<int32_t> b32(bounds.begin(), bounds.end());
    CG_CUDA(cudaMemcpyAsync(d_bounds, b32.data(), sizeof(int32_t) * (k + 1),
                            cudaMemcpyHostToDevice, s));
    CG_CUDA(cudaStreamSynchronize(s));  // b32 is a host temporary
  }
  const int words = (k + 31) / 32;
  const size_t sb_bytes = sizeof(int32_t) * (size_t)((k + 1 + 3) & ~3);
  const int grid_rows = grid_for((int64_t)V * 32, kBuildThreads, 16);

  // A
  int32_t* nseg = nullptr;
  int64_t* pos = nullptr;
  CG_CUDA(tmp.get(&nseg, V));
  CG_CUDA(tmp.get(&pos, (size_t)V + 1));
  row_nseg_kernel<<<grid_rows, kBuildThreads, sb_bytes + sizeof(uint32_t) * kBuildWarps * words,
                    s>>>(offsets, src, V, d_bounds, k, nseg);
  CG_LAUNCH_CHECK();
  CG_TRY(exclusive_scan_i32_to_i64(nseg, pos, V, s));
  int64_t npairs = 0;
  CG_CUDA(cudaMemcpyAsync(&npairs, pos + V, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  if (npairs >= 0x7FFFFFFF) {
    set_error("pr_build_segments: %lld subgraph rows exceed the int32 range", (long long)npairs);
    return CG_ERR_UNSUPPORTED;
  }
  g->rows = npairs;

  // B
  uint32_t* pseg = nullptr;
  uint32_t* sseg = nullptr;
  int32_t *prow = nullptr, *pcnt = nullptr, *piota = nullptr, *perm = nullptr, *inv = nullptr;
  int32_t* rowlen = nullptr;
  int64_t* rp = nullptr;
  CG_CUDA(tmp.get(&pseg, npairs));
  CG_CUDA(tmp.get(&sseg, npairs));
  CG_CUDA(tmp.get(&prow, npairs));
  CG_CUDA(tmp.get(&pcnt, npairs));
  CG_CUDA(tmp.get(&piota, npairs));
  CG_CUDA(tmp.get(&perm, npairs));
  CG_CUDA(tmp.get(&inv, npairs));
  CG_CUDA(tmp.get(&rowlen, npairs));
  CG_CUDA(tmp.get(&rp, (size_t)npairs + 1));
  row_pairs_kernel<<<grid_rows, kBuildThreads,
                     sb_bytes + sizeof(int32_t) * kBuildWarps * k +
                         sizeof(uint32_t) * kBuildWarps * words,
                     s>>>(offsets, src, V, d_bounds, k, pos, pseg, prow, pcnt);
  CG_LAUNCH_CHECK();

  // C
  int bits = 0;
  while ((1 << bits) < k) ++bits;
  if (npairs > 0) {
    iota_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(piota, npairs);
    CG_LAUNCH_CHECK();
    CG_TRY(radix_sort_pairs(pseg, piota, sseg, perm, npairs, bits > 0 ? bits : 1, s));
  }
  CG_CUDA(cudaMalloc((void**)&g->idx_map, sizeof(int32_t) * (size_t)(npairs > 0 ? npairs : 1)));
  if (npairs > 0) {
    pairs_to_rows_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(perm, prow, pcnt, npairs,
                                                                g->idx_map, rowlen, inv);
    CG_LAUNCH_CHECK();
  }
  CG_TRY(exclusive_scan_i32_to_i64(rowlen, rp, npairs, s));
  CG_CUDA(cudaMalloc((void**)&g->row_ptr, sizeof(int32_t) * (size_t)(npairs + 1)));
  to_i32_kernel<<<grid_for(npairs + 1, 256), 256, 0, s>>>(rp, npairs + 1, g->row_ptr);
  CG_LAUNCH_CHECK();
  int64_t* d_rb = nullptr;
  CG_CUDA(tmp.get(&d_rb, k + 1));
  segment_starts_kernel<<<(k + 1 + 127) / 128, 128, 0, s>>>(sseg, npairs, k, d_rb);
  CG_LAUNCH_CHECK();
  g->row_base.assign(k + 1, 0);
  CG_CUDA(cudaMemcpyAsync(g->row_base.data(), d_rb, sizeof(int64_t) * (k + 1),
                          cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  g->edge_base.assign(k + 1, 0);
  for (int q = 0; q <= k; ++q) {
    CG_CUDA(cudaMemcpyAsync(&g->edge_base[q], rp + g->row_base[q], sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
  }

  // D
  int32_t* col = nullptr;
  CG_CUDA(tmp.get(&col, (size_t)(E > 0 ? E : 1)));
  if (E > 0) {
    const size_t smem = sizeof(int64_t) * kBuildWarps * k + sizeof(int32_t) * (k + 1);
    scatter_edges_kernel<<<grid_rows, kBuildThreads, smem, s>>>(offsets, src, V, d_bounds, k, pos,
                                                                pseg, inv, rp, col);
    CG_LAUNCH_CHECK();
  }

  // E
  g->nb = (int32_t)ceil_div(V, B);
  {
    const size_t nbk = (size_t)k * (g->nb + 1);
    int32_t* blk_sm = nullptr;  // segment-major while it is built
    CG_CUDA(cudaMalloc((void**)&g->blk, sizeof(int32_t) * nbk));
    CG_CUDA(cudaMallocAsync((void**)&blk_sm, sizeof(int32_t) * nbk, s));
    blk_prefill_kernel<<<grid_for((int64_t)nbk, 256), 256, 0, s>>>(d_rb, k, g->nb, blk_sm);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess && npairs > 0) {
      blk_rows_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(d_rb, k, g->idx_map, npairs, B,
                                                            g->nb, blk_sm);
      ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
      blk_transpose_kernel<<<grid_for((int64_t)nbk, 256), 256, 0, s>>>(blk_sm, k, g->nb, g->blk);
      ce = cudaGetLastError();
    }
    cudaFreeAsync(blk_sm, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "pr_build_segments", __FILE__, __LINE__);
  }

  // F
  CG_CUDA(cudaStreamSynchronize(s));  // edge_base copies have landed
  CG_TRY(seg_plan_build(col, rp, g->row_ptr, npairs, E, k, g->row_base, g->edge_base, bounds,
                        &g->plan, s));
  CG_CUDA(cudaMalloc(&g->interm, sizeof(float) * (size_t)(npairs > 0 ? npairs : 1)));
  CG_CUDA(cudaMalloc((void**)&g->partials, sizeof(double) * 2 * (size_t)g->nb));
  CG_CUDA(cudaMalloc((void**)&g->counter, sizeof(unsigned)));
  CG_CUDA(cudaMemsetAsync(g->counter, 0, sizeof(unsigned), s));
  CG_CUDA(cudaMalloc((void**)&g->dslot, sizeof(double) * 4));
  CG_CUDA(cudaMemsetAsync(g->dslot, 0, sizeof(double) * 4, s));
  CG_CUDA(cudaMalloc((void**)&g->rank_tmp, sizeof(float) * (size_t)V));
  CG_CUDA(cudaMalloc((void**)&g->contrib_tmp, sizeof(float) * (size_t)V));
  CG_CUDA(cudaStreamSynchronize(s));
  g->bytes = 4 * (npairs + 1) + 4 * npairs + 4 * (int64_t)k * (g->nb + 1) +
             seg_plan_bytes(g->plan) + 4 * npairs + 16 * (int64_t)g->nb + 4 + 32 + 8 * (int64_t)V;
  return CG_OK;
}

void free_segmented(cg_segmented* g) {
  cudaFree(g->row_ptr);
  cudaFree(g->idx_map);
  cudaFree(g->blk);
  seg_plan_free(&g->plan);
  cudaFree(g->interm);
  cudaFree(g->partials);
  cudaFree(g->counter);
  cudaFree(g->dslot);
  cudaFree(g->rank_tmp);
  cudaFree(g->contrib_tmp);
}

}  // namespace

int validate_csr(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E,
                 cudaStream_t s) {
  unsigned long long* bad = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&bad, sizeof(unsigned long long), s));
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
  unsigned long long h = 0;
  if (e == cudaSuccess) {
    validate_csr_kernel<<<grid_for(std::max<int64_t>(V, E), 256), 256, 0, s>>>(offsets, src, V,
                                                                              E, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(bad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "validate_csr", __FILE__, __LINE__);
  if (h) {
    set_error("invalid CSR: %llu violations (offsets must rise from 0 to E; sources in [0, V))",
              h);
    return CG_ERR_INVALID_ARG;
  }
  return CG_OK;
}

}  // namespace cg

using namespace cg;

extern "C" {

int pr_build_segments(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E,
                      int32_t k, const int64_t* host_bounds, int32_t B, cg_segmented** out,
                      cudaStream_t stream) {
  CG_ARG(out != nullptr, "pr_build_segments: out is NULL");
  *out = nullptr;
  CG_ARG(V >= 1, "pr_build_segments: V must be >= 1 (got %d)", V);
  CG_ARG(E >= 0 && E < 0x7FFFFFFFLL, "pr_build_segments: E must be in [0, 2^31-1)");
  CG_ARG(offsets && (E == 0 || src), "pr_build_segments: null CSR pointer");
  CG_ARG(k >= 1 && k <= kMaxSegments, "pr_build_segments: num_segments must be in [1, %d]",
         kMaxSegments);
  CG_ARG(B >= 1 && B <= 6144, "pr_build_segments: merge_block must be in [1, 6144]");
  std::vector<int64_t> bounds(k + 1);
  if (host_bounds) {
    for (int q = 0; q <= k; ++q) bounds[q] = host_bounds[q];
    CG_ARG(bounds[0] == 0 && bounds[k] == V, "pr_build_segments: bounds must run from 0 to V");
    for (int q = 0; q < k; ++q)
      CG_ARG(bounds[q] <= bounds[q + 1], "pr_build_segments: bounds must be non-decreasing");
  } else {
    const int64_t N = ceil_div(V, k);
    for (int q = 0; q <= k; ++q) bounds[q] = std::min<int64_t>((int64_t)q * N, V);
  }
  CG_TRY(validate_csr(offsets, src, V, E, stream));
  cg_segmented* g = new cg_segmented();
  CG_CUDA(cudaGetDevice(&g->device));
  g->V = V;
  g->E = E;
  g->k = k;
  g->B = B;
  g->bounds = bounds;
  int st = build_impl(offsets, src, V, E, k, bounds, B, g, stream);
  if (st != CG_OK) {
    cudaStreamSynchronize(stream);
    free_segmented(g);
    delete g;
    return st;
  }
  *out = g;
  return CG_OK;
}

int cg_segmented_get_info(const cg_segmented* g, cg_segmented_info* info) {
  CG_ARG(g && info, "cg_segmented_get_info: null pointer");
  info->V = g->V;
  info->E = g->E;
  info->num_segments = g->k;
  info->merge_block = g->B;
  info->num_blocks = g->nb;
  info->rows = g->rows;
  info->q = g->V ? (double)g->rows / (double)g->V : 0.0;
  info->device_bytes = g->bytes;
  info->gather_tiles = g->plan.nchunks;
  info->table_vertices = g->plan.tab_cap;
  info->staged_segments = g->plan.m;
  info->staged_edges = g->plan.m > 0 ? g->edge_base[g->plan.m] : 0;
  info->ctas_per_sm = g->plan.ctas_per_sm;
  info->gather_threads = g->plan.threads;
  info->gather_overlap = g->plan.overlap;
  info->affine_segments = g->plan.m2 - g->plan.m;
  info->affine_edges = g->plan.m2 > g->plan.m ? g->edge_base[g->plan.m2] - g->edge_base[g->plan.m]
                                              : 0;
  return CG_OK;
}

int cg_segmented_stats(const cg_segmented* g, int64_t* q_rows_total, double* q,
                       size_t* device_bytes) {
  CG_ARG(g != nullptr, "cg_segmented_stats: null handle");
  if (q_rows_total) *q_rows_total = g->rows;
  if (q) *q = g->V ? (double)g->rows / (double)g->V : 0.0;
  if (device_bytes) *device_bytes = (size_t)g->bytes;
  return CG_OK;
}

int pr_set_gather_config(cg_segmented* g, int32_t threads, int32_t ctas_per_sm,
                         int32_t table_vertices, cudaStream_t stream) {
  CG_ARG(g != nullptr, "pr_set_gather_config: null handle");
  CG_ARG(table_vertices >= -1, "pr_set_gather_config: table_vertices must be >= -1");
  return seg_plan_configure(&g->plan, threads, ctas_per_sm, table_vertices, stream);
}

int pr_set_gather_overlap(cg_segmented* g, int32_t cached_warps, cudaStream_t stream) {
  CG_ARG(g != nullptr, "pr_set_gather_overlap: null handle");
  CG_ARG(cached_warps >= 0 && cached_warps <= 24,
         "pr_set_gather_overlap: cached_warps must be in [0, 24] (got %d)", cached_warps);
  const int before = g->plan.overlap_request;
  g->plan.overlap_request = cached_warps;
  const int rc = seg_plan_configure(&g->plan, g->plan.threads, g->plan.ctas_per_sm,
                                    g->plan.table_request, stream);
  if (rc != CG_OK) {  // keep the previous, valid configuration
    g->plan.overlap_request = before;
    seg_plan_configure(&g->plan, g->plan.threads, g->plan.ctas_per_sm, g->plan.table_request,
                       stream);
  }
  return rc;
}

int pr_set_gather_affine(cg_segmented* g, double head_min_avg_degree, cudaStream_t stream) {
  CG_ARG(g != nullptr, "pr_set_gather_affine: null handle");
  CG_ARG(head_min_avg_degree >= 0.0, "pr_set_gather_affine: head_min_avg_degree must be >= 0");
  const double before = g->plan.affine_head;
  g->plan.affine_head = head_min_avg_degree;
  const int rc = seg_plan_configure(&g->plan, g->plan.threads, g->plan.ctas_per_sm,
                                    g->plan.table_request, stream);
  if (rc != CG_OK) {  // keep the previous, valid configuration
    g->plan.affine_head = before;
    seg_plan_configure(&g->plan, g->plan.threads, g->plan.ctas_per_sm, g->plan.table_request,
                       stream);
  }
  return rc;
}

int pr_gather_table_capacity(int32_t ctas_per_sm) { return seg_table_capacity(ctas_per_sm); }

int pr_plan_bounds(const int32_t* dev_outdeg, int32_t V, int32_t smem_vertices,
                   double min_avg_degree, int32_t max_global_vertices, int32_t k_max,
                   int64_t* host_bounds, int32_t* k_out, cudaStream_t stream) {
  CG_ARG(dev_outdeg && host_bounds && k_out && V >= 1, "pr_plan_bounds: bad arguments");
  CG_ARG(k_max >= 1 && k_max <= kMaxSegments, "pr_plan_bounds: k_max must be in [1, %d]",
         kMaxSegments);
  if (max_global_vertices <= 0) {  // half of this GPU's L2 in 4-byte source values
    DeviceInfo di{};
    CG_TRY(device_info(&di));
    max_global_vertices = (int32_t)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)(di.l2_bytes / 8), (int64_t)0x7FFFFFFF));
  }
  if (smem_vertices < 0) smem_vertices = seg_table_capacity(1);
  std::vector<int32_t> deg(V);
  CG_CUDA(cudaMemcpyAsync(deg.data(), dev_outdeg, sizeof(int32_t) * (size_t)V,
                          cudaMemcpyDeviceToHost, stream));
  CG_CUDA(cudaStreamSynchronize(stream));
  std::vector<int64_t> b = {0};
  int64_t lo = 0;
  if (smem_vertices > 0) {
    while (lo < V && (int)b.size() < k_max) {
      const int64_t n = std::min<int64_t>(smem_vertices, V - lo);
      int64_t edges = 0;
      for (int64_t u = lo; u < lo + n; ++u) edges += deg[u];
      if ((double)edges < min_avg_degree * (double)n) break;
      lo += n;
      b.push_back(lo);
    }
  }
  if (lo < V) {
    // sources without out-edges at the end of the range (all of them, after
    // clustering) form one segment of their own: it has no edges to cut
    int64_t end = V;
    while (end > lo && deg[end - 1] == 0) --end;
    const int64_t left_k = k_max - ((int64_t)b.size() - 1) - (end < V && end > lo ? 1 : 0);
    if (left_k < 1) {
      b.back() = V;  // no room: the last shared-memory segment absorbs the rest
    } else {
      if (end > lo) {
        int64_t parts = std::max<int64_t>(1, ceil_div(end - lo, max_global_vertices));
        if (parts > left_k) parts = left_k;
        const int64_t step = ceil_div(end - lo, parts);
        for (int64_t q = 1; q <= parts; ++q) b.push_back(std::min<int64_t>(end, lo + q * step));
      }
      if (b.back() < V) b.push_back(V);
    }
  }
  *k_out = (int32_t)(b.size() - 1);
  for (size_t q = 0; q < b.size(); ++q) host_bounds[q] = b[q];
  return CG_OK;
}

int cg_segmented_export(const cg_segmented* g, int64_t* h_bounds, int64_t* h_row_base,
                        int64_t* h_edge_base, int64_t* d_row_ptr, int32_t* d_col,
                        int32_t* d_idx_map, int32_t* d_block_start, cudaStream_t s) {
  CG_ARG(g != nullptr, "cg_segmented_export: null handle");
  for (int q = 0; q <= g->k; ++q) {
    if (h_bounds) h_bounds[q] = g->bounds[q];
    if (h_row_base) h_row_base[q] = g->row_base[q];
    if (h_edge_base) h_edge_base[q] = g->edge_base[q];
  }
  if (d_row_ptr) {
    to_i64_kernel<<<grid_for(g->rows + 1, 256), 256, 0, s>>>(g->row_ptr, g->rows + 1, d_row_ptr);
    CG_LAUNCH_CHECK();
  }
  if (d_col && g->E > 0) CG_TRY(seg_plan_export_col(g->plan, g->row_ptr, d_col, s));
  if (d_idx_map && g->rows > 0)
    CG_CUDA(cudaMemcpyAsync(d_idx_map, g->idx_map, sizeof(int32_t) * g->rows,
                            cudaMemcpyDeviceToDevice, s));
  if (d_block_start) {
    int64_t* d_rb = nullptr;
    CG_CUDA(cudaMallocAsync((void**)&d_rb, sizeof(int64_t) * (g->k + 1), s));
    cudaError_t e = cudaMemcpyAsync(d_rb, g->row_base.data(), sizeof(int64_t) * (g->k + 1),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      blk_local_kernel<<<grid_for((int64_t)g->k * (g->nb + 1), 256), 256, 0, s>>>(
          g->blk, d_rb, g->k, g->nb, d_block_start);
      e = cudaGetLastError();
    }
    cudaFreeAsync(d_rb, s);
    if (e != cudaSuccess) return cuda_fail(e, "cg_segmented_export", __FILE__, __LINE__);
  }
  CG_CUDA(cudaStreamSynchronize(s));
  return CG_OK;
}

int cg_segmented_destroy(cg_segmented* g) {
  if (!g) return CG_OK;
  int cur = 0;
  const int dev = g->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  free_segmented(g);
  delete g;
  if (cur != dev) cudaSetDevice(cur);
  return CG_OK;
}

}  // extern "C"
