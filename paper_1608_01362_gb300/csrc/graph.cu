// Degrees, frequency-based clustering and CSR renumbering (Section V).
#include "common.cuh"

namespace cg {
namespace {

// Out-degree by counting sources; equal sources inside a warp are combined
// first (match_any) so hub vertices do not serialise on one atomic.
__global__ void out_degree_kernel(const int32_t* __restrict__ src, int64_t E, int32_t V,
                                  int32_t* __restrict__ outdeg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < E; base += stride) {
    const int64_t e = base + threadIdx.x;
    int32_t u = e < E ? __ldcs(src + e) : -1;
    if (u >= V) u = -1;  // out-of-range sources are ignored
    const unsigned key = u >= 0 ? (unsigned)u : (0x80000000u | (unsigned)lane);
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (u >= 0 && lane == __ffs(peers) - 1) atomicAdd(outdeg + u, __popc(peers));
  }
}

__global__ void inv_outdeg_kernel(const int32_t* __restrict__ outdeg, int32_t V,
                                  float* __restrict__ inv) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = outdeg[v];
    inv[v] = d > 0 ? 1.0f / (float)d : 0.0f;
  }
}

// Sort key: hotter (larger degree key) first -> ascending (INT32_MAX - key).
__global__ void cluster_key_kernel(const int32_t* __restrict__ outdeg, int32_t V, int32_t thr,
                                   uint32_t* __restrict__ key, int32_t* __restrict__ val) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t d = outdeg[v];
    if (d < 0) d = 0;
    key[v] = (uint32_t)(0x7FFFFFFF - d / thr);
    val[v] = (int32_t)v;
  }
}

__global__ void invert_perm_kernel(const int32_t* __restrict__ old_of_new, int32_t V,
                                   int32_t* __restrict__ new_of_old) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (int64_t)gridDim.x * blockDim.x)
    new_of_old[old_of_new[n]] = (int32_t)n;
}

__global__ void relabel_len_kernel(const int64_t* __restrict__ offsets,
                                   const int32_t* __restrict__ old_of_new, int32_t V,
                                   int64_t* __restrict__ len) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = old_of_new[n];
    len[n] = (o >= 0 && o < V) ? offsets[o + 1] - offsets[o] : 0;
  }
}

// One warp copies one new row: the old row's sources mapped to new IDs.
__global__ void relabel_copy_kernel(const int64_t* __restrict__ offsets,
                                    const int32_t* __restrict__ src,
                                    const int32_t* __restrict__ new_of_old,
                                    const int32_t* __restrict__ old_of_new, int32_t V,
                                    const int64_t* __restrict__ out_offsets,
                                    int32_t* __restrict__ out_src) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t n = warp; n < V; n += nwarps) {
    const int64_t o = old_of_new[n];
    if (o < 0 || o >= V) continue;  // not a permutation entry: row left empty
    const int64_t lo = offsets[o], hi = offsets[o + 1];
    const int64_t dst = out_offsets[n];
    for (int64_t e = lo + lane; e < hi; e += 32) {
      const int32_t u = __ldcs(src + e);
      out_src[dst + (e - lo)] = (u >= 0 && u < V) ? new_of_old[u] : u;
    }
  }
}

// Rows of w 16-byte words: out[i] = in[idx[i]] (zeros where idx[i] is out of range).
__global__ void permute_rows_kernel(const uint4* __restrict__ in, const int32_t* __restrict__ idx,
                                    int64_t n, int64_t n_in, int w, uint4* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * w;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / w, c = t - i * w;
    const int32_t j = idx[i];
    out[t] = (j >= 0 && j < n_in) ? in[(int64_t)j * w + c] : make_uint4(0u, 0u, 0u, 0u);
  }
}

template <typename W>
__global__ void permute_kernel(const W* __restrict__ in, const int32_t* __restrict__ idx,
                               int64_t n, int64_t n_in, W* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = idx[i];
    out[i] = (j >= 0 && j < n_in) ? in[j] : W(0);
  }
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int cg_out_degree(const int32_t* src, int64_t E, int32_t V, int32_t* outdeg,
                  cudaStream_t stream) {
  CG_ARG(V >= 1, "cg_out_degree: V must be >= 1 (got %d)", V);
  CG_ARG(E >= 0, "cg_out_degree: E must be >= 0");
  CG_ARG(outdeg && (E == 0 || src), "cg_out_degree: null pointer");
  CG_CUDA(cudaMemsetAsync(outdeg, 0, sizeof(int32_t) * (size_t)V, stream));
  if (E == 0) return CG_OK;
  out_degree_kernel<<<grid_for(E, 256), 256, 0, stream>>>(src, E, V, outdeg);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int cg_inv_outdeg(const int32_t* outdeg, int32_t V, float* inv, cudaStream_t stream) {
  CG_ARG(V >= 1 && outdeg && inv, "cg_inv_outdeg: bad arguments");
  inv_outdeg_kernel<<<grid_for(V, 256), 256, 0, stream>>>(outdeg, V, inv);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int cg_cluster(const int32_t* outdeg, int32_t V, int64_t E, int32_t mode, int32_t* new_of_old,
               int32_t* old_of_new, cudaStream_t stream) {
  CG_ARG(V >= 1 && E >= 0, "cg_cluster: V must be >= 1 and E >= 0");
  CG_ARG(outdeg && new_of_old && old_of_new, "cg_cluster: null pointer");
  CG_ARG(mode == 0 || mode == 1, "cg_cluster: mode must be 0 or 1 (got %d)", mode);
  CG_ARG(new_of_old != old_of_new, "cg_cluster: outputs must not alias");
  int64_t thr = 1;
  if (mode == 1) {
    thr = E / V;
    if (thr < 1) thr = 1;
    if (thr > 0x7FFFFFFF) thr = 0x7FFFFFFF;
  }
  uint32_t* key = nullptr;
  uint32_t* key2 = nullptr;
  int32_t* val = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&key, sizeof(uint32_t) * (size_t)V * 2, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&val, sizeof(int32_t) * (size_t)V, stream);
  if (e != cudaSuccess) {
    if (key) cudaFreeAsync(key, stream);
    return cuda_fail(e, "cg_cluster scratch", __FILE__, __LINE__);
  }
  key2 = key + V;
  int st = CG_OK;
  cluster_key_kernel<<<grid_for(V, 256), 256, 0, stream>>>(outdeg, V, (int32_t)thr, key, val);
  e = cudaGetLastError();
  if (e != cudaSuccess) st = cuda_fail(e, "cluster_key", __FILE__, __LINE__);
  if (st == CG_OK) st = radix_sort_pairs(key, val, key2, old_of_new, V, 31, stream);
  if (st == CG_OK) {
    invert_perm_kernel<<<grid_for(V, 256), 256, 0, stream>>>(old_of_new, V, new_of_old);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "invert_perm", __FILE__, __LINE__);
  }
  cudaFreeAsync(key, stream);
  cudaFreeAsync(val, stream);
  return st;
}

int cg_permute4(const void* in, int64_t n_in, const int32_t* idx, int64_t n, void* out,
                cudaStream_t stream) {
  CG_ARG(n >= 0 && n_in >= 0, "cg_permute4: negative size");
  if (n == 0) return CG_OK;
  CG_ARG(in && idx && out && in != out, "cg_permute4: null or aliased pointer");
  permute_kernel<uint32_t><<<grid_for(n, 256), 256, 0, stream>>>((const uint32_t*)in, idx, n,
                                                                 n_in, (uint32_t*)out);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int cg_permute8(const void* in, int64_t n_in, const int32_t* idx, int64_t n, void* out,
                cudaStream_t stream) {
  CG_ARG(n >= 0 && n_in >= 0, "cg_permute8: negative size");
  if (n == 0) return CG_OK;
  CG_ARG(in && idx && out && in != out, "cg_permute8: null or aliased pointer");
  CG_ARG(((uintptr_t)in & 7) == 0 && ((uintptr_t)out & 7) == 0,
         "cg_permute8: buffers must be 8-byte aligned");
  permute_kernel<uint64_t><<<grid_for(n, 256), 256, 0, stream>>>((const uint64_t*)in, idx, n,
                                                                 n_in, (uint64_t*)out);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int cg_permute_rows(const void* in, int64_t n_in, int32_t row_bytes, const int32_t* idx,
                    int64_t n, void* out, cudaStream_t stream) {
  CG_ARG(n >= 0 && n_in >= 0, "cg_permute_rows: negative size");
  CG_ARG(row_bytes > 0 && row_bytes % 16 == 0, "cg_permute_rows: row_bytes must be a positive "
         "multiple of 16 (got %d)", row_bytes);
  if (n == 0) return CG_OK;
  CG_ARG(in && idx && out && in != out, "cg_permute_rows: null or aliased pointer");
  CG_ARG(((uintptr_t)in | (uintptr_t)out) % 16 == 0, "cg_permute_rows: rows need 16-byte "
         "aligned buffers");
  const int w = row_bytes / 16;
  permute_rows_kernel<<<grid_for(n * w, 256), 256, 0, stream>>>((const uint4*)in, idx, n, n_in, w,
                                                                (uint4*)out);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int cg_relabel_csr(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E,
                   const int32_t* new_of_old, const int32_t* old_of_new, int64_t* out_offsets,
                   int32_t* out_src, cudaStream_t stream) {
  CG_ARG(V >= 1 && E >= 0, "cg_relabel_csr: V must be >= 1 and E >= 0");
  CG_ARG(offsets && new_of_old && old_of_new && out_offsets && (E == 0 || (src && out_src)),
         "cg_relabel_csr: null pointer");
  CG_ARG((E == 0 || (const void*)out_src != (const void*)src) &&
             (const void*)out_offsets != (const void*)offsets,
         "cg_relabel_csr: outputs must not alias inputs");
  int64_t* len = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&len, sizeof(int64_t) * ((size_t)V + 1), stream));
  int st = CG_OK;
  relabel_len_kernel<<<grid_for(V, 256), 256, 0, stream>>>(offsets, old_of_new, V, len);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) st = cuda_fail(e, "relabel_len", __FILE__, __LINE__);
  if (st == CG_OK) st = exclusive_scan_i64(len, out_offsets, V, stream);
  if (st == CG_OK && E > 0) {
    relabel_copy_kernel<<<grid_for((int64_t)V * 32, 256), 256, 0, stream>>>(
        offsets, src, new_of_old, old_of_new, V, out_offsets, out_src);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "relabel_copy", __FILE__, __LINE__);
  }
  cudaFreeAsync(len, stream);
  return st;
}

}  // extern "C"
