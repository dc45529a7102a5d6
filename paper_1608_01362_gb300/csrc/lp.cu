// Label propagation over the segmented graph (the paper's LP application,
// Table IV): synchronous passes L'[v] = min(L[v], min over in-neighbours u of
// L[u]) -- Algorithm 3's gather with a min, Algorithm 4's merge with a min,
// fused with the label update and a count of changed labels.  Integer
// arithmetic throughout: results are exact.
#include "handles.cuh"
#include "update.cuh"

namespace cg {
namespace {

// Merge of one warp-owned block with the min operator (same walk as the
// PageRank merge), then L' = min(L, acc) and the number of changed labels.
__global__ void __launch_bounds__(kMergeWarps * 32)
lp_merge_update_kernel(const int32_t* __restrict__ blk, const int32_t* __restrict__ idx_map,
                       const int32_t* __restrict__ interm, int k, int nb, int B, int32_t V,
                       const int32_t* __restrict__ labels_in, int32_t* __restrict__ labels_out,
                       unsigned long long* __restrict__ changed) {
  extern __shared__ int32_t lp_acc_all[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mb = (int64_t)blockIdx.x * kMergeWarps + w;
  if (mb >= nb) return;
  int32_t* acc = lp_acc_all + (int64_t)w * B;
  const int64_t v0 = mb * B;
  const int n = (int)((V - v0) < B ? (V - v0) : B);
  warp_merge<MinI32>(blk, idx_map, interm, k, nb, mb, v0, n, acc);
  unsigned long long cnt = 0;
  constexpr int U = 4;  // labels per lane loaded together
  for (int i0 = lane; i0 < n; i0 += 32 * U) {
    int32_t old[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      old[u] = i0 + 32 * u < n ? __ldcs(labels_in + v0 + i0 + 32 * u) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + 32 * u;
      if (i < n) {
        const int32_t l = acc[i] < old[u] ? acc[i] : old[u];
        __stcs(labels_out + v0 + i, l);
        cnt += (l != old[u]);
      }
    }
  }
  cnt = warp_sum(cnt);
  if (lane == 0 && cnt) atomicAdd(changed, cnt);
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int lp_iterate(const cg_segmented* g, const int32_t* labels_in, int32_t* labels_out,
               int64_t* dev_changed, int64_t* host_changed, cudaStream_t stream) {
  CG_ARG(g && labels_in && labels_out, "lp_iterate: null argument");
  CG_ARG(labels_in != labels_out, "lp_iterate: labels_out must not alias labels_in");
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(dev_changed);
  if (!cnt) cnt = reinterpret_cast<unsigned long long*>(g->dslot + 3);
  CG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), stream));
  CG_TRY(run_seg_gather<MinI32>(g->plan, labels_in, g->V, (int32_t*)g->interm, stream));
  const size_t smem = (size_t)kMergeWarps * g->B * 4;
  if (smem > 32 * 1024)
    CG_CUDA(cudaFuncSetAttribute((const void*)lp_merge_update_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  lp_merge_update_kernel<<<(unsigned)ceil_div(g->nb, kMergeWarps), kMergeWarps * 32, smem,
                           stream>>>(g->blk, g->idx_map, (const int32_t*)g->interm, g->k, g->nb,
                                     g->B, g->V, labels_in, labels_out, cnt);
  CG_LAUNCH_CHECK();
  if (host_changed) {
    unsigned long long h = 0;
    CG_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CG_CUDA(cudaStreamSynchronize(stream));
    *host_changed = (int64_t)h;
  }
  return CG_OK;
}

int lp_run(const cg_segmented* g, int32_t* labels, int64_t max_passes, int64_t* host_passes,
           int64_t* host_changes, cudaStream_t stream) {
  CG_ARG(g && labels && host_passes, "lp_run: null argument");
  CG_ARG(max_passes >= 1, "lp_run: max_passes must be >= 1");
  int32_t* a = labels;
  int32_t* b = reinterpret_cast<int32_t*>(g->rank_tmp);  // V int32 of handle scratch
  int64_t p = 0;
  for (; p < max_passes;) {
    int64_t changed = 0;
    CG_TRY(lp_iterate(g, a, b, nullptr, &changed, stream));
    if (host_changes) host_changes[p] = changed;
    ++p;
    int32_t* t = a;
    a = b;
    b = t;
    if (changed == 0) break;
  }
  if (a != labels)
    CG_CUDA(cudaMemcpyAsync(labels, a, sizeof(int32_t) * (size_t)g->V, cudaMemcpyDeviceToDevice,
                            stream));
  CG_CUDA(cudaStreamSynchronize(stream));
  *host_passes = p;
  return CG_OK;
}

}  // extern "C"
