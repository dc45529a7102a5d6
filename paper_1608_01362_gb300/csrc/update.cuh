// The PageRank vertex update (Algorithm 5's VertexUpdate in normalised form)
// shared by the segmented and the plain paths, with the FP64 dangling-mass
// and residual reductions.
#pragma once

#include "common.cuh"

namespace cg {
namespace {

constexpr int kMergeWarps = 8;  // warps per merge / update block

struct PrArgs {
  const float* inv;
  const float* rank_in;
  float* rank_out;
  float* contrib_out;
  float base;      // (1-d)/V
  float d;         // damping
  double inv_V;    // 1/V
  const double* D_in;
  double* D_out;
  double* resid_out;
  double* partials;
  unsigned* counter;
  int32_t V;
};

// Vertex update (Algorithm 5's VertexUpdate, normalised) for one warp's
// destinations [v0, v0+n) with sums in acc; returns the warp's FP64 partial
// sums of the dangling mass and of the L1 residual (valid in lane 0).
__device__ __forceinline__ void warp_vertex_update(const float* acc, int64_t v0, int n,
                                                   const PrArgs& a, float Dv, double* dsum,
                                                   double* rsum) {
  const int lane = threadIdx.x & 31;
  float dpart = 0.0f, rpart = 0.0f;  // <= B/32 terms per lane, then FP64
  for (int i = lane; i < n; i += 32) {
    const int64_t v = v0 + i;
    const float r = a.base + a.d * (acc[i] + Dv);
    const float iv = __ldcs(a.inv + v);
    const float old = __ldcs(a.rank_in + v);
    __stcs(a.rank_out + v, r);
    __stcs(a.contrib_out + v, r * iv);
    if (iv == 0.0f) dpart += r;
    rpart += fabsf(r - old);
  }
  *dsum = warp_sum((double)dpart);
  *rsum = warp_sum((double)rpart);
}

// Per-block FP64 partials, then the last block to finish reduces all
// partials in a fixed order (no float atomics: deterministic).
__device__ __forceinline__ void block_finish(double dsum, double rsum, const PrArgs& a) {
  __shared__ double s_d[kMergeWarps], s_r[kMergeWarps];
  __shared__ double sh[32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_d[w] = dsum;
    s_r[w] = rsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bd = 0.0, br = 0.0;
    for (int q = 0; q < kMergeWarps; ++q) {
      bd += s_d[q];
      br += s_r[q];
    }
    a.partials[2 * blockIdx.x] = bd;
    a.partials[2 * blockIdx.x + 1] = br;
    __threadfence();
    const unsigned prev = atomicAdd(a.counter, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double sd = 0.0, sr = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += kMergeWarps * 32) {
      sd += __ldcg(a.partials + 2 * q);
      sr += __ldcg(a.partials + 2 * q + 1);
    }
    sd = block_sum<double, kMergeWarps * 32>(sd, sh);
    sr = block_sum<double, kMergeWarps * 32>(sr, sh);
    if (threadIdx.x == 0) {
      *a.D_out = sd;
      if (a.resid_out) *a.resid_out = sr;
      *a.counter = 0u;
    }
  }
}

// Plain path: the gathered sums are already dense.
__global__ void __launch_bounds__(kMergeWarps * 32)
dense_update_kernel(const float* __restrict__ sums, int B, int nb, PrArgs a) {
  extern __shared__ float acc_all[];
  const double D = *a.D_in;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mb = (int64_t)blockIdx.x * kMergeWarps + w;
  double dsum = 0.0, rsum = 0.0;
  if (mb < nb) {
    float* acc = acc_all + (int64_t)w * B;
    const int64_t v0 = mb * B;
    const int n = (int)((a.V - v0) < B ? (a.V - v0) : B);
    for (int i = lane; i < n; i += 32) acc[i] = __ldcs(sums + v0 + i);
    __syncwarp();
    warp_vertex_update(acc, v0, n, a, (float)(D * a.inv_V), &dsum, &rsum);
  }
  block_finish(dsum, rsum, a);
}

}  // namespace
}  // namespace cg
