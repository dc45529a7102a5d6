// PageRank through the segmented graph (Algorithms 3, 4 and 5) and the plain
// pull baseline (Algorithm 1), plus the stand-alone gather / merge entry
// points.
//
// One iteration of pr_iterate = two kernels (+ a tiny carry fix-up):
//   gather_tile_kernel   Algorithm 3 over every subgraph, segments in order
//                        (tiles are dispatched in segment order, so the
//                        random reads of contrib stay inside one segment's
//                        slice at a time), writing intermBuf sequentially;
//   merge_update_kernel  Algorithm 4 per block of B destinations: the block's
//                        rows of every subgraph are added, segment by
//                        segment, into a shared-memory accumulator; then the
//                        vertex update of Algorithm 5 and the FP64 partial
//                        sums of the dangling mass and of the L1 residual;
//                        the last block to finish reduces the partials in a
//                        fixed order (no float atomics: deterministic).
#include "handles.cuh"
#include "update.cuh"

namespace cg {
namespace {

// Cache-aware merge (Algorithm 4) fused with the vertex update.
__global__ void __launch_bounds__(kMergeWarps * 32, 6)
merge_update_kernel(const int32_t* __restrict__ blk, const int32_t* __restrict__ idx_map,
                    const float* __restrict__ interm, int k, int nb, int B, PrArgs a) {
  extern __shared__ float acc_all[];
  const double D = *a.D_in;
  const int w = threadIdx.x >> 5;
  const int64_t mb = (int64_t)blockIdx.x * kMergeWarps + w;
  double dsum = 0.0, rsum = 0.0;
  if (mb < nb) {
    float* acc = acc_all + (int64_t)w * B;
    const int64_t v0 = mb * B;
    const int n = (int)((a.V - v0) < B ? (a.V - v0) : B);
    warp_merge<SumF32>(blk, idx_map, interm, k, nb, mb, v0, n, acc);
    warp_vertex_update(acc, v0, n, a, D, &dsum, &rsum);
  }
  block_finish(dsum, rsum, a);
}

// Generic merge (Algorithm 4 alone) with identity fill.
template <class Op>
__global__ void __launch_bounds__(kMergeWarps * 32)
merge_only_kernel(const int32_t* __restrict__ blk, const int32_t* __restrict__ idx_map,
                  const typename Op::T* __restrict__ interm, int k, int nb, int B, int32_t V,
                  typename Op::T* __restrict__ out) {
  using T = typename Op::T;
  extern __shared__ unsigned char raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mb = (int64_t)blockIdx.x * kMergeWarps + w;
  if (mb >= nb) return;
  T* acc = reinterpret_cast<T*>(raw) + (int64_t)w * B;
  const int64_t v0 = mb * B;
  const int n = (int)((V - v0) < B ? (V - v0) : B);
  warp_merge<Op>(blk, idx_map, interm, k, nb, mb, v0, n, acc);
  for (int i = lane; i < n; i += 32) out[v0 + i] = acc[i];
}

__global__ void pr_init_kernel(const float* __restrict__ inv, int32_t V, float* __restrict__ rank,
                               float* __restrict__ contrib, unsigned long long* __restrict__ ndang) {
  const float r = 1.0f / (float)V;
  unsigned long long c = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const float iv = inv[v];
    rank[v] = r;
    contrib[v] = r * iv;
    c += iv == 0.0f;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(ndang, c);
}

// Personalised start: all mass on the seed; D = the seed's mass if it is
// dangling.
__global__ void ppr_init_kernel(const float* __restrict__ inv, int32_t V, int32_t seed,
                                float* __restrict__ rank, float* __restrict__ contrib,
                                double* __restrict__ D) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const float r = v == seed ? 1.0f : 0.0f;
    rank[v] = r;
    contrib[v] = r * inv[v];
    if (v == seed) *D = inv[v] == 0.0f ? 1.0 : 0.0;
  }
}

__global__ void pr_init_finish_kernel(const unsigned long long* __restrict__ ndang, int32_t V,
                                      double* __restrict__ D) {
  *D = (double)(*ndang) * (double)(1.0f / (float)V);
}

// contrib = rank * inv and per-block FP64 partials of the dangling mass.
__global__ void pr_contrib_kernel(const float* __restrict__ inv, const float* __restrict__ rank,
                                  int32_t V, float* __restrict__ contrib,
                                  double* __restrict__ partials) {
  __shared__ double sh[32];
  double d = 0.0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const float iv = inv[v], r = rank[v];
    contrib[v] = r * iv;
    if (iv == 0.0f) d += (double)r;
  }
  d = block_sum<double, 256>(d, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = d;
}

__global__ void sum_partials_kernel(const double* __restrict__ partials, int n,
                                    double* __restrict__ out) {
  __shared__ double sh[32];
  double d = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) d += partials[i];
  d = block_sum<double, 256>(d, sh);
  if (threadIdx.x == 0) *out = d;
}

int set_merge_smem(const void* fn, size_t bytes) {
  // the kernels also hold a little static shared memory, so opt in above 32 KB
  if (bytes > 32 * 1024)
    CG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return CG_OK;
}

struct IterBufs {
  const float* rank_in;
  const float* contrib_in;
  float* rank_out;
  float* contrib_out;
  const double* D_in;
  double* D_out;
  double* resid;
};

// Buffers of iteration t out of T: results land in (rank_out, contrib_out)
// after the last iteration; intermediate iterations alternate with tmp.
IterBufs iter_bufs(int t, int T, const float* rank_in, const float* contrib_in, float* rank_out,
                   float* contrib_out, float* rank_tmp, float* contrib_tmp, double* D_io,
                   double* dslot, double* resid) {
  IterBufs b;
  auto dst_is_out = [&](int it) { return ((T - 1 - it) % 2) == 0; };
  if (t == 0) {
    b.rank_in = rank_in;
    b.contrib_in = contrib_in;
    b.D_in = D_io;
  } else {
    const bool prev_out = dst_is_out(t - 1);
    b.rank_in = prev_out ? rank_out : rank_tmp;
    b.contrib_in = prev_out ? contrib_out : contrib_tmp;
    b.D_in = dslot + ((t - 1) & 1);
  }
  b.rank_out = dst_is_out(t) ? rank_out : rank_tmp;
  b.contrib_out = dst_is_out(t) ? contrib_out : contrib_tmp;
  b.D_out = (t == T - 1) ? D_io : dslot + (t & 1);
  b.resid = resid ? resid + t : dslot + 2;
  return b;
}

int check_pr_args(int32_t V, const float* inv, const float* rank_in, const float* contrib_in,
                  float* rank_out, float* contrib_out, double damping, int32_t iterations,
                  double* D_io) {
  CG_ARG(inv && rank_in && contrib_in && rank_out && contrib_out && D_io,
         "pagerank: null pointer argument");
  CG_ARG(iterations >= 1, "pagerank: iterations must be >= 1 (got %d)", iterations);
  CG_ARG(damping >= 0.0 && damping <= 1.0, "pagerank: damping must be in [0, 1]");
  CG_ARG(rank_out != rank_in && contrib_out != contrib_in && (const float*)rank_out != contrib_in &&
             (const float*)contrib_out != rank_in && rank_out != contrib_out,
         "pagerank: output vectors must not alias the inputs or each other");
  (void)V;
  return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int pr_init(const float* inv, int32_t V, float* rank, float* contrib, double* D,
            cudaStream_t stream) {
  CG_ARG(V >= 1 && inv && rank && contrib && D, "pr_init: bad arguments");
  unsigned long long* nd = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&nd, sizeof(unsigned long long), stream));
  cudaError_t e = cudaMemsetAsync(nd, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    pr_init_kernel<<<grid_for(V, 256), 256, 0, stream>>>(inv, V, rank, contrib, nd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    pr_init_finish_kernel<<<1, 1, 0, stream>>>(nd, V, D);
    e = cudaGetLastError();
  }
  cudaFreeAsync(nd, stream);
  if (e != cudaSuccess) return cuda_fail(e, "pr_init", __FILE__, __LINE__);
  return CG_OK;
}

int pr_contrib(const float* inv, const float* rank, int32_t V, float* contrib, double* D,
               cudaStream_t stream) {
  CG_ARG(V >= 1 && inv && rank && contrib && D, "pr_contrib: bad arguments");
  CG_ARG((const float*)contrib != rank && (const float*)contrib != inv,
         "pr_contrib: contrib must not alias the inputs");
  const int grid = grid_for(V, 256, 4);
  double* part = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * grid, stream));
  pr_contrib_kernel<<<grid, 256, 0, stream>>>(inv, rank, V, contrib, part);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    sum_partials_kernel<<<1, 256, 0, stream>>>(part, grid, D);
    e = cudaGetLastError();
  }
  cudaFreeAsync(part, stream);
  if (e != cudaSuccess) return cuda_fail(e, "pr_contrib", __FILE__, __LINE__);
  return CG_OK;
}

int cg_seg_gather_phases(const cg_segmented* g, int32_t op, const void* x, void* interm,
                         int32_t phases, cudaStream_t stream) {
  CG_ARG(g && x, "cg_seg_gather_phases: null argument");
  CG_ARG(phases >= 0 && phases <= kPhaseAll, "cg_seg_gather_phases: phases must be in [0, 7]");
  if (!interm) interm = g->interm;
  if (op == CG_OP_SUM_F32)
    return run_seg_gather<SumF32>(g->plan, (const float*)x, g->V, (float*)interm, stream,
                                  phases);
  if (op == CG_OP_MIN_I32)
    return run_seg_gather<MinI32>(g->plan, (const int32_t*)x, g->V, (int32_t*)interm, stream,
                                  phases);
  set_error("cg_seg_gather_phases: unknown op %d", op);
  return CG_ERR_INVALID_ARG;
}

int cg_seg_gather(const cg_segmented* g, int32_t op, const void* x, void* interm,
                  cudaStream_t stream) {
  CG_ARG(g && x, "cg_seg_gather: null argument");
  if (!interm) interm = g->interm;
  if (op == CG_OP_SUM_F32)
    return run_seg_gather<SumF32>(g->plan, (const float*)x, g->V, (float*)interm, stream);
  if (op == CG_OP_MIN_I32)
    return run_seg_gather<MinI32>(g->plan, (const int32_t*)x, g->V, (int32_t*)interm, stream);
  set_error("cg_seg_gather: unknown op %d", op);
  return CG_ERR_INVALID_ARG;
}

int merge(const cg_segmented* g, int32_t op, const void* interm, void* out, cudaStream_t stream) {
  CG_ARG(g && out && (interm || g->rows == 0), "merge: null argument");
  const unsigned grid = (unsigned)ceil_div(g->nb, kMergeWarps);
  const size_t smem = (size_t)kMergeWarps * g->B * 4;
  if (op == CG_OP_SUM_F32) {
    auto fn = merge_only_kernel<SumF32>;
    CG_TRY(set_merge_smem((const void*)fn, smem));
    fn<<<grid, kMergeWarps * 32, smem, stream>>>(g->blk, g->idx_map, (const float*)interm, g->k,
                                                 g->nb, g->B, g->V, (float*)out);
  } else if (op == CG_OP_MIN_I32) {
    auto fn = merge_only_kernel<MinI32>;
    CG_TRY(set_merge_smem((const void*)fn, smem));
    fn<<<grid, kMergeWarps * 32, smem, stream>>>(g->blk, g->idx_map, (const int32_t*)interm,
                                                 g->k, g->nb, g->B, g->V, (int32_t*)out);
  } else {
    set_error("merge: unknown op %d", op);
    return CG_ERR_INVALID_ARG;
  }
  CG_LAUNCH_CHECK();
  return CG_OK;
}

static int merge_update_seeded(const cg_segmented* g, const float* inv, const float* rank_in,
                               float* rank_out, float* contrib_out, double damping,
                               const double* D_in, double* D_out, double* resid_out,
                               int32_t seed, cudaStream_t stream);

int pr_merge_update(const cg_segmented* g, const float* inv, const float* rank_in,
                    float* rank_out, float* contrib_out, double damping, const double* D_in,
                    double* D_out, double* resid_out, cudaStream_t stream) {
  return merge_update_seeded(g, inv, rank_in, rank_out, contrib_out, damping, D_in, D_out,
                             resid_out, -1, stream);
}

static int merge_update_seeded(const cg_segmented* g, const float* inv, const float* rank_in,
                               float* rank_out, float* contrib_out, double damping,
                               const double* D_in, double* D_out, double* resid_out,
                               int32_t seed, cudaStream_t stream) {
  CG_ARG(g && inv && rank_in && rank_out && contrib_out && D_in && D_out,
         "pr_merge_update: null argument");
  CG_ARG(damping >= 0.0 && damping <= 1.0, "pr_merge_update: damping must be in [0, 1]");
  CG_ARG(rank_out != rank_in && (const float*)contrib_out != rank_in && rank_out != contrib_out,
         "pr_merge_update: outputs must not alias the inputs or each other");
  const size_t smem = (size_t)kMergeWarps * g->B * 4;
  CG_TRY(set_merge_smem((const void*)merge_update_kernel, smem));
  PrArgs a;
  a.inv = inv;
  a.rank_in = rank_in;
  a.rank_out = rank_out;
  a.contrib_out = contrib_out;
  a.base = (float)((1.0 - damping) / (double)g->V);
  a.d = (float)damping;
  a.inv_V = 1.0 / (double)g->V;
  a.D_in = D_in;
  a.D_out = D_out;
  a.resid_out = resid_out;
  a.partials = g->partials;
  a.counter = g->counter;
  a.V = g->V;
  a.seed = seed;
  merge_update_kernel<<<(unsigned)ceil_div(g->nb, kMergeWarps), kMergeWarps * 32, smem,
                        stream>>>(g->blk, g->idx_map, (const float*)g->interm, g->k, g->nb,
                                  g->B, a);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

static int iterate_seeded(const cg_segmented* g, const float* inv, const float* rank_in,
                          const float* contrib_in, float* rank_out, float* contrib_out,
                          double damping, int32_t iterations, double* D_io, double* resid,
                          int32_t seed, cudaStream_t stream) {
  CG_TRY(check_pr_args(g->V, inv, rank_in, contrib_in, rank_out, contrib_out, damping,
                       iterations, D_io));
  for (int t = 0; t < iterations; ++t) {
    IterBufs b = iter_bufs(t, iterations, rank_in, contrib_in, rank_out, contrib_out,
                           g->rank_tmp, g->contrib_tmp, D_io, g->dslot, resid);
    CG_TRY(run_seg_gather<SumF32>(g->plan, b.contrib_in, g->V, (float*)g->interm, stream));
    CG_TRY(merge_update_seeded(g, inv, b.rank_in, b.rank_out, b.contrib_out, damping, b.D_in,
                               b.D_out, b.resid, seed, stream));
  }
  return CG_OK;
}

int pr_iterate(const cg_segmented* g, const float* inv, const float* rank_in,
               const float* contrib_in, float* rank_out, float* contrib_out, double damping,
               int32_t iterations, double* D_io, double* resid, cudaStream_t stream) {
  CG_ARG(g != nullptr, "pr_iterate: null handle");
  return iterate_seeded(g, inv, rank_in, contrib_in, rank_out, contrib_out, damping, iterations,
                        D_io, resid, -1, stream);
}

int pr_init_ppr(const float* inv, int32_t V, int32_t seed, float* rank, float* contrib,
                double* D, cudaStream_t stream) {
  CG_ARG(V >= 1 && inv && rank && contrib && D, "pr_init_ppr: bad arguments");
  CG_ARG(seed >= 0 && seed < V, "pr_init_ppr: seed %d outside [0, %d)", seed, V);
  ppr_init_kernel<<<grid_for(V, 256), 256, 0, stream>>>(inv, V, seed, rank, contrib, D);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int pr_iterate_ppr(const cg_segmented* g, const float* inv, const float* rank_in,
                   const float* contrib_in, float* rank_out, float* contrib_out, double damping,
                   int32_t iterations, int32_t seed, double* D_io, double* resid,
                   cudaStream_t stream) {
  CG_ARG(g != nullptr, "pr_iterate_ppr: null handle");
  CG_ARG(seed >= 0 && seed < g->V, "pr_iterate_ppr: seed %d outside [0, %d)", seed, g->V);
  return iterate_seeded(g, inv, rank_in, contrib_in, rank_out, contrib_out, damping, iterations,
                        D_io, resid, seed, stream);
}

// ------------------------------------------------------------------ plain

int pr_plain_create(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E,
                    cg_plain** out, cudaStream_t stream) {
  CG_ARG(out != nullptr, "pr_plain_create: out is NULL");
  *out = nullptr;
  CG_ARG(V >= 1 && E >= 0 && E < 0x7FFFFFFFLL, "pr_plain_create: V >= 1 and 0 <= E < 2^31-1");
  CG_ARG(offsets && (E == 0 || src), "pr_plain_create: null CSR pointer");
  CG_TRY(validate_csr(offsets, src, V, E, stream));
  cg_plain* p = new cg_plain();
  CG_CUDA(cudaGetDevice(&p->device));
  p->V = V;
  p->E = E;
  p->offsets = offsets;
  p->src = src;
  p->nb = (int32_t)ceil_div(ceil_div(V, 512), kMergeWarps);  // update blocks
  int st = plan_tiles<int64_t>(offsets + 1, V, E, &p->plan, stream);
  cudaError_t e = cudaSuccess;
  if (st == CG_OK) e = cudaMalloc((void**)&p->acc, sizeof(float) * (size_t)V);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->partials, sizeof(double) * 2 * p->nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->counter, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(p->counter, 0, sizeof(unsigned), stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->dslot, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dslot, 0, sizeof(double) * 4, stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->rank_tmp, sizeof(float) * (size_t)V);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->contrib_tmp, sizeof(float) * (size_t)V);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (st == CG_OK && e != cudaSuccess) st = cuda_fail(e, "pr_plain_create", __FILE__, __LINE__);
  if (st != CG_OK) {
    pr_plain_destroy(p);
    return st;
  }
  p->bytes = tile_plan_bytes(p->plan) + 12 * (int64_t)V + 16 * (int64_t)p->nb + 36;
  *out = p;
  return CG_OK;
}

int pr_plain_destroy(cg_plain* p) {
  if (!p) return CG_OK;
  int cur = 0;
  const int dev = p->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  free_tile_plan(&p->plan);
  cudaFree(p->acc);
  cudaFree(p->partials);
  cudaFree(p->counter);
  cudaFree(p->dslot);
  cudaFree(p->rank_tmp);
  cudaFree(p->contrib_tmp);
  delete p;
  if (cur != dev) cudaSetDevice(cur);
  return CG_OK;
}

int pr_iterate_plain(const cg_plain* p, const float* inv, const float* rank_in,
                     const float* contrib_in, float* rank_out, float* contrib_out,
                     double damping, int32_t iterations, double* D_io, double* resid,
                     int32_t probe, cudaStream_t stream) {
  CG_ARG(p != nullptr, "pr_iterate_plain: null handle");
  CG_TRY(check_pr_args(p->V, inv, rank_in, contrib_in, rank_out, contrib_out, damping,
                       iterations, D_io));
  const int B = 512;
  const int nb = (int)ceil_div(p->V, B);
  const size_t smem = (size_t)kMergeWarps * B * 4;
  CG_TRY(set_merge_smem((const void*)dense_update_kernel, smem));
  for (int t = 0; t < iterations; ++t) {
    IterBufs b = iter_bufs(t, iterations, rank_in, contrib_in, rank_out, contrib_out,
                           p->rank_tmp, p->contrib_tmp, D_io, p->dslot, resid);
    if (probe)
      CG_TRY((run_tile_gather<SumF32, true, int64_t>(p->plan, p->offsets + 1, p->src, b.contrib_in,
                                                p->V, p->acc, stream)));
    else
      CG_TRY((run_tile_gather<SumF32, false, int64_t>(p->plan, p->offsets + 1, p->src, b.contrib_in,
                                                 p->V, p->acc, stream)));
    PrArgs a;
    a.inv = inv;
    a.rank_in = b.rank_in;
    a.rank_out = b.rank_out;
    a.contrib_out = b.contrib_out;
    a.base = (float)((1.0 - damping) / (double)p->V);
    a.d = (float)damping;
    a.inv_V = 1.0 / (double)p->V;
    a.D_in = b.D_in;
    a.D_out = b.D_out;
    a.resid_out = b.resid;
    a.partials = p->partials;
    a.counter = p->counter;
    a.V = p->V;
    a.seed = -1;
    dense_update_kernel<<<(unsigned)ceil_div(nb, kMergeWarps), kMergeWarps * 32, smem,
                          stream>>>(p->acc, B, nb, a);
    CG_LAUNCH_CHECK();
  }
  return CG_OK;
}

}  // extern "C"
