// Device-wide exclusive scan and stable LSD radix sort used by the
// preprocessing steps (clustering, segment construction).  Plain three-phase
// designs with no inter-block waiting: reduce tiles -> scan tile sums
// (recursively) -> scan tiles with their offsets.
#include "common.cuh"

namespace cg {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename TI>
__global__ void tile_reduce_kernel(const TI* __restrict__ in, int64_t n,
                                   int64_t* __restrict__ sums) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
    if (i < n) acc += (int64_t)in[i];
  }
  acc = block_sum<int64_t, kScanThreads>(acc, sh);
  if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

// Exclusive scan of one tile per block; each thread owns kScanItems
// consecutive items.  tile_off: exclusive offsets of the tiles (or NULL for a
// single tile).  out[n] receives the grand total (written by the last tile).
template <typename TI>
__global__ void tile_scan_kernel(const TI* __restrict__ in, int64_t n,
                                 const int64_t* __restrict__ tile_off,
                                 int64_t* __restrict__ out) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t tsum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t i = base + j;
    v[j] = i < n ? (int64_t)in[i] : 0;
    tsum += v[j];
  }
  // block exclusive scan of per-thread sums
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  int64_t wbase = 0, total = 0;
  for (int q = 0; q < kScanThreads / 32; ++q) {
    if (q < w) wbase += warp_tot[q];
    total += warp_tot[q];
  }
  int64_t run = (tile_off ? tile_off[blockIdx.x] : 0) + wbase + incl - tsum;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t i = base + j;
    if (i < n) out[i] = run;
    run += v[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    out[n] = (tile_off ? tile_off[blockIdx.x] : 0) + total;
}

template <typename TI>
int exclusive_scan_impl(const TI* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    CG_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return CG_OK;
  }
  const int64_t tiles = ceil_div(n, kScanTile);
  if (tiles == 1) {
    tile_scan_kernel<TI><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    CG_LAUNCH_CHECK();
    return CG_OK;
  }
  int64_t* buf = nullptr;  // tile sums [tiles], tile offsets [tiles+1]
  CG_CUDA(cudaMallocAsync((void**)&buf, sizeof(int64_t) * (2 * tiles + 1), s));
  tile_reduce_kernel<TI><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, buf);
  int st = CG_OK;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) st = cuda_fail(e, "tile_reduce", __FILE__, __LINE__);
  if (st == CG_OK) st = exclusive_scan_impl<int64_t>(buf, buf + tiles, tiles, s);
  if (st == CG_OK) {
    tile_scan_kernel<TI><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, buf + tiles, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "tile_scan", __FILE__, __LINE__);
  }
  cudaFreeAsync(buf, s);
  return st;
}

// ---------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;                       // items per thread
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096
constexpr int kSortWarps = kSortThreads / 32;

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                  int32_t* __restrict__ counts, int64_t ntiles) {
  __shared__ int32_t h[256];
  for (int i = threadIdx.x; i < 256; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int j = 0; j < kSortRounds; ++j) {
    int64_t i = base + (int64_t)j * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += kSortThreads)
    counts[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Stable scatter of one tile: warp w owns items [w*512, w*512+512) of the
// tile, visited in rounds of 32 consecutive items, so (warp, round, lane)
// order is the input order.  Equal digits are ranked with __match_any_sync.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin,
                                     const int32_t* __restrict__ vin, int64_t n, int shift,
                                     const int64_t* __restrict__ offs, int64_t ntiles,
                                     uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int32_t wc[kSortWarps][256];
  for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * (kSortRounds * 32);
  uint32_t k[kSortRounds];
  int32_t v[kSortRounds];
  int32_t lr[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * 32 + lane;
    const bool ok = i < n;
    k[r] = ok ? kin[i] : 0u;
    v[r] = ok ? vin[i] : 0;
    const unsigned d = (k[r] >> shift) & 255u;
    const unsigned key = ok ? d : (0x100u | (unsigned)lane);  // unique for idle lanes
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    lr[r] = ok ? wc[w][d] + __popc(peers & lt) : 0;
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) wc[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kSortThreads) {
    int32_t run = 0;
    for (int q = 0; q < kSortWarps; ++q) {
      int32_t t = wc[q][d];
      wc[q][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * 32 + lane;
    if (i < n) {
      const unsigned d = (k[r] >> shift) & 255u;
      const int64_t pos = offs[(int64_t)d * ntiles + blockIdx.x] + wc[w][d] + lr[r];
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
  }
}

}  // namespace

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return exclusive_scan_impl<int64_t>(in, out, n, s);
}
int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return exclusive_scan_impl<int32_t>(in, out, n, s);
}

int radix_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_out,
                     int32_t* vals_out, int64_t n, int bits, cudaStream_t s) {
  if (n <= 0) return CG_OK;
  const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
  const int64_t ntiles = ceil_div(n, kSortTile);
  uint32_t* kb = nullptr;
  int32_t* vb = nullptr;
  int32_t* counts = nullptr;
  int64_t* offs = nullptr;
  int st = CG_OK;
  cudaError_t e;
  e = cudaMallocAsync((void**)&kb, sizeof(uint32_t) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&vb, sizeof(int32_t) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&counts, sizeof(int32_t) * 256 * ntiles, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&offs, sizeof(int64_t) * (256 * ntiles + 1), s);
  if (e != cudaSuccess) st = cuda_fail(e, "radix scratch", __FILE__, __LINE__);
  // ping-pong so that the last pass lands in (keys_out, vals_out)
  const uint32_t* ksrc = keys_in;
  const int32_t* vsrc = vals_in;
  for (int p = 0; p < passes && st == CG_OK; ++p) {
    // passes alternate between the scratch pair and the output pair, ending in the output
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* kdst = to_out ? keys_out : kb;
    int32_t* vdst = to_out ? vals_out : vb;
    radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ksrc, n, 8 * p, counts, ntiles);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = cuda_fail(e, "radix_hist", __FILE__, __LINE__); break; }
    st = exclusive_scan_i32_to_i64(counts, offs, 256 * ntiles, s);
    if (st != CG_OK) break;
    radix_scatter_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ksrc, vsrc, n, 8 * p, offs,
                                                                    ntiles, kdst, vdst);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = cuda_fail(e, "radix_scatter", __FILE__, __LINE__); break; }
    ksrc = kdst;
    vsrc = vdst;
  }
  if (kb) cudaFreeAsync(kb, s);
  if (vb) cudaFreeAsync(vb, s);
  if (counts) cudaFreeAsync(counts, s);
  if (offs) cudaFreeAsync(offs, s);
  return st;
}

}  // namespace cg
