// The PageRank vertex update (Algorithm 5's VertexUpdate in normalised form)
// shared by the segmented and the plain paths, with the FP64 dangling-mass
// and residual reductions.
#pragma once

#include "gather.cuh"

namespace cg {
namespace {

constexpr int kMergeWarps = 8;  // warps per merge / update block

// ---------------------------------------------------------------------------
// Cache-aware merge (Algorithm 4).  Each warp owns one merge block of B
// destinations (a shared-memory accumulator of B values) and folds the
// block's rows [blk[b][s], blk[b+1][s]) of intermBuf (blk block-major) into
// acc[idx_map[i] - b*B], segment after segment in ascending order, so every
// destination receives its partial sums in segment order (deterministic).
//
// The rows of up to 32 segments are handled as one flattened sequence
// (segment-major, so flattened order is segment order): lane l holds the
// inclusive prefix of the row counts of segment s0+l, and a flattened
// position f belongs to the segment whose prefix first exceeds f (a binary
// search over the lanes).  A warp loads 32*U consecutive flattened rows at
// once, then applies them 32 at a time; inside one group of 32 lanes the rows
// of one segment have distinct destinations, and different segments are
// applied one after the other in ascending order.  An operator that is exact
// in any order (min) applies a whole group at once with shared-memory
// atomics instead.  A block whose segments hold a few rows each then costs
// one memory round trip instead of one per segment, and a hub block's
// segments with hundreds of rows keep 32*U loads in flight instead of 32.
// ---------------------------------------------------------------------------

template <class Op>
__device__ __forceinline__ void warp_merge(const int32_t* __restrict__ blk,
                                           const int32_t* __restrict__ idx_map,
                                           const typename Op::T* __restrict__ interm, int k,
                                           int nb, int64_t mb, int64_t v0, int n,
                                           typename Op::T* acc) {
  using T = typename Op::T;
  constexpr int U = 4;  // groups of 32 flattened rows loaded together
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < n; i += 32) acc[i] = Op::identity();
  __syncwarp();
  for (int s0 = 0; s0 < k; s0 += 32) {
    const int ls = s0 + lane;
    int32_t lo = 0, hi = 0;
    if (ls < k) {  // block-major: the lanes read consecutive words
      lo = __ldg(blk + mb * k + ls);
      hi = __ldg(blk + (mb + 1) * k + ls);
    }
    // inclusive prefix of the row counts over the lanes' segments
    int32_t pre = hi - lo;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(kFull, pre, o);
      if (lane >= o) pre += t;
    }
    const int32_t off = lo - (pre - (hi - lo));  // row index = flattened position + off
    const int32_t total = __shfl_sync(kFull, pre, 31);
    for (int32_t base = 0; base < total; base += 32 * U) {
      int32_t seg[U], dd[U];
      T xx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t f = base + u * 32 + lane;
        int j = 0;  // number of segments whose rows all precede f
#pragma unroll
        for (int step = 16; step; step >>= 1)
          if (__shfl_sync(kFull, pre, j + step - 1) <= f) j += step;
        const int32_t row = f + __shfl_sync(kFull, off, j);
        seg[u] = f < total ? j : 32;
        dd[u] = 0;
        xx[u] = Op::identity();
        if (f < total) {
          dd[u] = __ldcs(idx_map + row);
          xx[u] = __ldcs(interm + row);
        }
      }
      if constexpr (Op::kExactAnyOrder) {  // e.g. min: every row at once
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t lv = (int64_t)dd[u] - v0;
          if (seg[u] < 32 && (uint64_t)lv < (uint64_t)n) Op::atomic_op(acc + lv, xx[u]);
        }
        continue;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {  // apply in flattened (= segment) order
        unsigned pend = __ballot_sync(kFull, seg[u] < 32);
        while (pend) {
          const int sj = __shfl_sync(kFull, seg[u], __ffs(pend) - 1);
          const bool mine = seg[u] == sj;
          if (mine) {
            const int64_t lv = (int64_t)dd[u] - v0;
            if ((uint64_t)lv < (uint64_t)n) acc[lv] = Op::op(acc[lv], xx[u]);
          }
          __syncwarp();
          pend &= ~__ballot_sync(kFull, mine);
        }
      }
    }
  }
  __syncwarp();
}

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
  int32_t seed;    // -1: uniform teleport; else personalised to this vertex
};

// Vertex update (Algorithm 5's VertexUpdate, normalised) for one warp's
// destinations [v0, v0+n) with sums in acc; returns the warp's FP64 partial
// sums of the dangling mass and of the L1 residual (valid in lane 0).
__device__ __forceinline__ void warp_vertex_update(const float* acc, int64_t v0, int n,
                                                   const PrArgs& a, double Dfull, double* dsum,
                                                   double* rsum) {
  const float Dv = (float)(Dfull * a.inv_V);
  const int lane = threadIdx.x & 31;
  const float tele = (float)((1.0 - (double)a.d) + (double)a.d * Dfull);
  float dpart = 0.0f, rpart = 0.0f;  // <= B/32 terms per lane, then FP64
  constexpr int U = 8;  // destinations per lane whose inputs are loaded together
  for (int i0 = lane; i0 < n; i0 += 32 * U) {
    float iv[U], old[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + 32 * u;
      iv[u] = 0.0f;
      old[u] = 0.0f;
      if (i < n) {
        iv[u] = __ldcs(a.inv + v0 + i);
        old[u] = __ldcs(a.rank_in + v0 + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + 32 * u;
      if (i < n) {
        const int64_t v = v0 + i;
        float r;
        if (a.seed < 0) {
          r = a.base + a.d * (acc[i] + Dv);
        } else {  // personalised: teleport and dangling mass return to the seed
          r = a.d * acc[i];
          if (v == a.seed) r += tele;
        }
        __stcs(a.rank_out + v, r);
        __stcs(a.contrib_out + v, r * iv[u]);
        if (iv[u] == 0.0f) dpart += r;
        rpart += fabsf(r - old[u]);
      }
    }
  }
  // the lanes' partials: summed in FP32 over groups of 2o lanes as long as a
  // group's sum stays within 256 ranks (each lane holds at most ceil(n/32)),
  // then the groups in FP64 (FP64 runs at a small fraction of the FP32 rate)
  const int per_lane = (n + 31) >> 5;
  int o = 16;
  while (o >= 1 && 2 * o * per_lane > 256) o >>= 1;
  for (int f = o; f >= 1; f >>= 1) {
    dpart += __shfl_down_sync(0xffffffffu, dpart, f);
    rpart += __shfl_down_sync(0xffffffffu, rpart, f);
  }
  double dd = (double)dpart, rr = (double)rpart;
  for (int f = 16; f > o; f >>= 1) {
    dd += __shfl_down_sync(0xffffffffu, dd, f);
    rr += __shfl_down_sync(0xffffffffu, rr, f);
  }
  *dsum = dd;
  *rsum = rr;
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
    warp_vertex_update(acc, v0, n, a, D, &dsum, &rsum);
  }
  block_finish(dsum, rsum, a);
}

}  // namespace
}  // namespace cg
