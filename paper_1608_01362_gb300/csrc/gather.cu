// Host side of the gather: tiling plans, launch configuration, launches.
#include <algorithm>

#include "gather.cuh"

namespace cg {

int gather_table_capacity(int ctas) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  int sm_smem = 0, reserved = 0, optin = 0;
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ctas < 1) ctas = 1;
  int64_t per = (int64_t)sm_smem / ctas - reserved;
  if (per > optin) per = optin;
  const int64_t dyn = per - kGatherStaticSmem - 2 * (int64_t)kGatherPadTile * 4;
  if (dyn <= 0) return 0;
  return (int)((dyn / 4) & ~31LL);
}

static size_t dyn_smem_bytes(const GatherPlan& p) {
  return (size_t)(p.tab_cap + 2 * kGatherPadTile) * 4;
}

template <class Op, bool PROBE, typename RowEndT>
static const void* kernel_ptr() {
  return (const void*)gather_kernel<Op, kGatherThreads, kGatherIPT, PROBE, RowEndT>;
}

int configure_gather(GatherPlan* p, int tab_vertices, int ctas_per_sm, cudaStream_t s) {
  if (ctas_per_sm < 1) ctas_per_sm = 1;
  const int cap = gather_table_capacity(ctas_per_sm);
  int tab = tab_vertices < 0 ? cap : std::min(tab_vertices, cap);
  tab &= ~3;
  p->tab_cap = tab;
  p->ctas_per_sm = ctas_per_sm;
  std::vector<int32_t> lo(p->k > 0 ? p->k : 1), tn(p->k > 0 ? p->k : 1);
  for (int q = 0; q < p->k; ++q) {
    lo[q] = (int32_t)p->src_bounds[q];
    tn[q] = (int32_t)std::min<int64_t>(tab, p->src_bounds[q + 1] - p->src_bounds[q]);
  }
  if (p->k > 0) {
    CG_CUDA(cudaMemcpyAsync(p->seg_lo, lo.data(), sizeof(int32_t) * p->k, cudaMemcpyHostToDevice,
                            s));
    CG_CUDA(cudaMemcpyAsync(p->seg_tab, tn.data(), sizeof(int32_t) * p->k,
                            cudaMemcpyHostToDevice, s));
    CG_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  p->grid = (int)std::min<int64_t>(std::max<int64_t>(p->ntiles, 1),
                                   (int64_t)di.sm_count * ctas_per_sm);
  return CG_OK;
}

template <typename RowEndT>
int plan_gather(const RowEndT* row_end, int64_t nrows, int64_t nedges, int k,
                const std::vector<int64_t>& row_base, const std::vector<int64_t>& edge_base,
                const std::vector<int64_t>& src_bounds, int tab_vertices, int ctas_per_sm,
                GatherPlan* p, cudaStream_t s) {
  p->nrows = nrows;
  p->nedges = nedges;
  p->tile = kGatherTile;
  p->k = k;
  p->src_bounds = src_bounds;
  std::vector<int64_t> tile_base(k + 1, 0), seg_diag(k + 1, 0);
  for (int q = 0; q < k; ++q) {
    const int64_t items = (row_base[q + 1] - row_base[q]) + (edge_base[q + 1] - edge_base[q]);
    tile_base[q + 1] = tile_base[q] + ceil_div(items, kGatherTile);
    seg_diag[q] = row_base[q] + edge_base[q];
  }
  seg_diag[k] = nrows + nedges;
  p->ntiles = tile_base[k];
  if (p->ntiles >= 0x7FFFFFFF) {
    set_error("gather plan: too many tiles");
    return CG_ERR_UNSUPPORTED;
  }
  const size_t nb = sizeof(int32_t) * (size_t)(p->ntiles + 1);
  CG_CUDA(cudaMalloc((void**)&p->tile_row, nb));
  CG_CUDA(cudaMalloc((void**)&p->tile_edge, nb));
  CG_CUDA(cudaMalloc((void**)&p->tile_seg, nb));
  CG_CUDA(cudaMalloc(&p->carry, nb));
  CG_CUDA(cudaMalloc((void**)&p->carry_row, nb));
  CG_CUDA(cudaMalloc((void**)&p->seg_lo, sizeof(int32_t) * (k > 0 ? k : 1)));
  CG_CUDA(cudaMalloc((void**)&p->seg_tab, sizeof(int32_t) * (k > 0 ? k : 1)));
  int64_t* d_meta = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&d_meta, sizeof(int64_t) * 2 * (k + 1), s));
  cudaError_t e = cudaMemcpyAsync(d_meta, tile_base.data(), sizeof(int64_t) * (k + 1),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_meta + k + 1, seg_diag.data(), sizeof(int64_t) * (k + 1),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    tile_partition_kernel<RowEndT><<<grid_for(p->ntiles + 1, 256), 256, 0, s>>>(
        row_end, nrows, nedges, kGatherTile, p->ntiles, k, d_meta, d_meta + k + 1, p->tile_row,
        p->tile_edge, p->tile_seg);
    e = cudaGetLastError();
  }
  cudaFreeAsync(d_meta, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors go out of scope
  if (e != cudaSuccess) return cuda_fail(e, "plan_gather", __FILE__, __LINE__);
  return configure_gather(p, tab_vertices, ctas_per_sm, s);
}

template int plan_gather<int32_t>(const int32_t*, int64_t, int64_t, int,
                                  const std::vector<int64_t>&, const std::vector<int64_t>&,
                                  const std::vector<int64_t>&, int, int, GatherPlan*,
                                  cudaStream_t);
template int plan_gather<int64_t>(const int64_t*, int64_t, int64_t, int,
                                  const std::vector<int64_t>&, const std::vector<int64_t>&,
                                  const std::vector<int64_t>&, int, int, GatherPlan*,
                                  cudaStream_t);

void free_plan(GatherPlan* p) {
  cudaFree(p->tile_row);
  cudaFree(p->tile_edge);
  cudaFree(p->tile_seg);
  cudaFree(p->carry);
  cudaFree(p->carry_row);
  cudaFree(p->seg_lo);
  cudaFree(p->seg_tab);
  *p = GatherPlan();
}

int64_t plan_bytes(const GatherPlan& p) { return 20 * (p.ntiles + 1) + 8 * (int64_t)p.k; }

template <class Op, bool PROBE, typename RowEndT>
int run_gather(const GatherPlan& p, const RowEndT* row_end, const int32_t* col,
               const typename Op::T* x, int32_t nx, typename Op::T* out, cudaStream_t s) {
  if (p.ntiles == 0) return CG_OK;
  const size_t smem = dyn_smem_bytes(p);
  auto fn = gather_kernel<Op, kGatherThreads, kGatherIPT, PROBE, RowEndT>;
  if (smem > 48 * 1024)
    CG_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  fn<<<p.grid, kGatherThreads, smem, s>>>(row_end, col, x, nx, p.tile_row, p.tile_edge,
                                          p.tile_seg, p.ntiles, p.seg_lo, p.seg_tab, p.tab_cap,
                                          out, reinterpret_cast<typename Op::T*>(p.carry),
                                          p.carry_row);
  CG_LAUNCH_CHECK();
  carry_fixup_kernel<Op><<<grid_for(p.ntiles, 256, 4), 256, 0, s>>>(
      reinterpret_cast<const typename Op::T*>(p.carry), p.carry_row, p.ntiles, p.nrows, out);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

template int run_gather<SumF32, false, int32_t>(const GatherPlan&, const int32_t*, const int32_t*,
                                                const float*, int32_t, float*, cudaStream_t);
template int run_gather<SumF32, false, int64_t>(const GatherPlan&, const int64_t*, const int32_t*,
                                                const float*, int32_t, float*, cudaStream_t);
template int run_gather<SumF32, true, int64_t>(const GatherPlan&, const int64_t*, const int32_t*,
                                               const float*, int32_t, float*, cudaStream_t);
template int run_gather<MinI32, false, int32_t>(const GatherPlan&, const int32_t*, const int32_t*,
                                                const int32_t*, int32_t, int32_t*, cudaStream_t);
template int run_gather<MinI32, false, int64_t>(const GatherPlan&, const int64_t*, const int32_t*,
                                                const int32_t*, int32_t, int32_t*, cudaStream_t);

}  // namespace cg
