// Collaborative filtering by gradient descent (the paper's CF application,
// Section VI / Table III) on a user-item rating graph.  One sweep updates
// both sides from the same old factors (Jacobi):
//   e_ui = r_ui - p_u . q_i
//   p_u += step ((1/deg u) sum_{i in N(u)} e_ui q_i - lambda p_u)
//   q_i += step ((1/deg i) sum_{u in N(i)} e_ui p_u - lambda q_i)
// and reports sum e_ui^2 of the old factors (FP64).
//
// Each side is a per-vertex gather of err * neighbour-row over that side's
// CSR (Algorithm 3's gather with a 32-wide row and a dot product per edge).
// On this GPU both factor matrices fit in L2 (Netflix shape: 61 MB of user
// rows and 2.3 MB of item rows in FP32, half that in BF16), so the source
// set is one segment and the gather is split only for load balance: every
// vertex's rating list is cut into pieces of at most kPiece ratings, a warp
// takes one piece at a time, and a group of K/8 lanes takes one rating (each
// lane 8 dimensions: 32 or 16 bytes of the row).  Piece partial gradients
// are summed per vertex, in piece order, by the update kernel.
//
// Storage precision of P and Q: FP32, BF16, or BF16 hi + lo pairs
// (hi = bf16(x), lo = bf16(x - hi), packed in one 32-bit word per entry);
// arithmetic is FP32, SSE is FP64.
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace cg {
constexpr int kCfPiece = 512;   // ratings per gather piece
constexpr int kCfWide = 64;     // vertices with more pieces are updated by a whole block
constexpr int kCfThreads = 256;
}  // namespace cg

struct cg_bipartite {
  int device = 0;
  int64_t U = 0, I = 0, R = 0;
  int32_t K = 32;
  int32_t precision = 0;
  const int64_t* uoff = nullptr;
  const int32_t* uitem = nullptr;
  const uint8_t* urate = nullptr;
  const int64_t* ioff = nullptr;
  const int32_t* iuser = nullptr;
  const uint8_t* irate = nullptr;
  // pieces per side: owning vertex, first rating; per vertex its first piece
  int32_t* pvtx[2] = {nullptr, nullptr};
  int64_t* pbeg[2] = {nullptr, nullptr};
  int64_t* poff[2] = {nullptr, nullptr};
  int64_t npieces[2] = {0, 0};
  float* gpart[2] = {nullptr, nullptr};  // [npieces][K] piece gradients
  int32_t* wide[2] = {nullptr, nullptr};  // vertices with more than kCfWide pieces
  int32_t nwide[2] = {0, 0};
  // factor storage (FP32, BF16, or BF16 hi + lo words); index 1 unused
  void* P[2] = {nullptr, nullptr};
  void* Q[2] = {nullptr, nullptr};
  double* partials = nullptr;  // [gather grid] SSE
  unsigned* counter = nullptr;
  int gather_grid = 0;
  int64_t bytes = 0;
};

namespace cg {
namespace {

__device__ __forceinline__ float b_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float b_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void unpack8(const uint4& h, float (&y)[8]) {
  y[0] = b_lo(h.x); y[1] = b_hi(h.x); y[2] = b_lo(h.y); y[3] = b_hi(h.y);
  y[4] = b_lo(h.z); y[5] = b_hi(h.z); y[6] = b_lo(h.w); y[7] = b_hi(h.w);
}

__device__ __forceinline__ uint32_t pk(float a, float b) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// 8 consecutive dimensions of row `row` (K per row) in the storage format.
// BF16 hi + lo is stored as one 32-bit word per dimension (hi in the low
// half, lo in the high half), so a row is one 128-byte line at K = 32, like
// FP32, and a lane reads its 8 dimensions with two 16-byte loads.
__device__ __forceinline__ float hilo(uint32_t w) { return b_lo(w) + b_hi(w); }

template <int PREC>
__device__ __forceinline__ void load8(const void* p0, int64_t row, int K, int d0, float (&y)[8]) {
  const int64_t at = row * K + d0;
  if (PREC == 0) {
    const float4* f = reinterpret_cast<const float4*>(static_cast<const float*>(p0) + at);
    const float4 a = __ldg(f), b = __ldg(f + 1);
    y[0] = a.x; y[1] = a.y; y[2] = a.z; y[3] = a.w;
    y[4] = b.x; y[5] = b.y; y[6] = b.z; y[7] = b.w;
  } else if (PREC == 1) {
    unpack8(__ldg(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(p0) + at)), y);
  } else {
    const uint4* f = reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(p0) + at);
    const uint4 a = __ldg(f), b = __ldg(f + 1);
    y[0] = hilo(a.x); y[1] = hilo(a.y); y[2] = hilo(a.z); y[3] = hilo(a.w);
    y[4] = hilo(b.x); y[5] = hilo(b.y); y[6] = hilo(b.z); y[7] = hilo(b.w);
  }
}

// hi = bf16(x), lo = bf16(x - hi) as one word (hi low, lo high)
__device__ __forceinline__ uint32_t pack_hilo(float x) {
  const uint32_t h = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
  const float hf = __uint_as_float(h << 16);
  const uint32_t l = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x - hf));
  return h | (l << 16);
}

template <int PREC>
__device__ __forceinline__ void store8(void* p0, int64_t row, int K, int d0, const float (&x)[8]) {
  const int64_t at = row * K + d0;
  if (PREC == 0) {
    float4* f = reinterpret_cast<float4*>(static_cast<float*>(p0) + at);
    f[0] = make_float4(x[0], x[1], x[2], x[3]);
    f[1] = make_float4(x[4], x[5], x[6], x[7]);
  } else if (PREC == 1) {
    uint32_t h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = pk(x[2 * q], x[2 * q + 1]);
    *reinterpret_cast<uint4*>(static_cast<uint16_t*>(p0) + at) = make_uint4(h[0], h[1], h[2], h[3]);
  } else {
    uint4* f = reinterpret_cast<uint4*>(static_cast<uint32_t*>(p0) + at);
    f[0] = make_uint4(pack_hilo(x[0]), pack_hilo(x[1]), pack_hilo(x[2]), pack_hilo(x[3]));
    f[1] = make_uint4(pack_hilo(x[4]), pack_hilo(x[5]), pack_hilo(x[6]), pack_hilo(x[7]));
  }
}

// ---------------------------------------------------------------------------
// Gather of one side: for every piece (vertex v, ratings [b, e)), the
// partial gradient sum_{ratings} e_r * y_nbr and (user side) sum e_r^2.
// LANES = K / 8 lanes per rating; 32 / LANES ratings per warp step.
// ---------------------------------------------------------------------------
template <int LANES, int PREC, bool SSE>
__global__ void __launch_bounds__(kCfThreads)
cf_gather_kernel(const int32_t* __restrict__ pvtx, const int64_t* __restrict__ pbeg,
                 const int64_t* __restrict__ off, int64_t npieces,
                 const int32_t* __restrict__ nbr, const uint8_t* __restrict__ rate,
                 const void* __restrict__ s0, const void* __restrict__ n0,
                 float* __restrict__ gpart, double* __restrict__ partials,
                 unsigned* __restrict__ counter, double* __restrict__ sse_out) {
  constexpr int K = 8 * LANES;
  constexpr int GROUPS = 32 / LANES;
  const int lane = threadIdx.x & 31;
  const int sub = lane % LANES, grp = lane / LANES;
  const int d0 = 8 * sub;
  const unsigned gmask = (LANES == 32 ? 0xffffffffu : ((1u << LANES) - 1u)) << (grp * LANES);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double sse_acc = 0.0;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npieces;
       p += nwarp) {
    const int32_t v = __ldg(pvtx + p);
    const int64_t b = __ldg(pbeg + p);
    const int64_t vend = __ldg(off + v + 1);
    const int64_t e_end = min(b + kCfPiece, vend);
    float x[8], g[8];
    load8<PREC>(s0, v, K, d0, x);
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = 0.0f;
    float se = 0.0f;
    for (int64_t r = b + grp; r < e_end; r += 2 * GROUPS) {
      // two ratings of this group in flight
      const int64_t r2 = r + GROUPS;
      const bool has2 = r2 < e_end;
      // the rating stream is read once: evict-first, so it does not push
      // factor rows out of L2
      const int32_t u1 = __ldcs(nbr + r);
      const int32_t u2 = has2 ? __ldcs(nbr + r2) : u1;
      const float rt1 = (float)__ldcs(rate + r);
      const float rt2 = has2 ? (float)__ldcs(rate + r2) : 0.0f;
      float y1[8], y2[8];
      load8<PREC>(n0, u1, K, d0, y1);
      load8<PREC>(n0, u2, K, d0, y2);
      float t1 = 0.0f, t2 = 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        t1 = fmaf(x[q], y1[q], t1);
        t2 = fmaf(x[q], y2[q], t2);
      }
#pragma unroll
      for (int o = 1; o < LANES; o <<= 1) {
        t1 += __shfl_xor_sync(gmask, t1, o);
        t2 += __shfl_xor_sync(gmask, t2, o);
      }
      const float e1 = rt1 - t1;
      const float e2 = has2 ? rt2 - t2 : 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) g[q] = fmaf(e1, y1[q], fmaf(e2, y2[q], g[q]));
      if (SSE && sub == 0) se = fmaf(e1, e1, fmaf(e2, e2, se));
    }
    // gradient: sum over the warp's groups (lanes with the same `sub`)
#pragma unroll
    for (int o = LANES; o < 32; o <<= 1)
#pragma unroll
      for (int q = 0; q < 8; ++q) g[q] += __shfl_xor_sync(0xffffffffu, g[q], o);
    if (grp == 0) {
      float4* dst = reinterpret_cast<float4*>(gpart + p * K + d0);
      dst[0] = make_float4(g[0], g[1], g[2], g[3]);
      dst[1] = make_float4(g[4], g[5], g[6], g[7]);
    }
    if (SSE) sse_acc += (double)warp_sum(se);
  }
  if (!SSE) return;
  __shared__ double sh[32];
  __shared__ bool s_last;
  const double bs = block_sum<double, kCfThreads>(lane == 0 ? sse_acc : 0.0, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kCfThreads) t += __ldcg(partials + i);
  t = block_sum<double, kCfThreads>(t, sh);
  if (threadIdx.x == 0) {
    if (sse_out) *sse_out = t;
    *counter = 0u;
  }
}

// x_v += step (g_v / deg v - lambda x_v), g_v = sum of v's piece gradients in
// piece order.  One group of LANES lanes per vertex.
template <int LANES, int PREC>
__global__ void __launch_bounds__(kCfThreads)
cf_update_kernel(const int64_t* __restrict__ poff, const int64_t* __restrict__ off, int64_t n,
                 const float* __restrict__ gpart, void* x0, float lambda, float step) {
  constexpr int K = 8 * LANES;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / LANES;
  const int sub = (int)(t % LANES);
  const int d0 = 8 * sub;
  for (int64_t v = t / LANES; v < n; v += ng) {
    if (poff[v + 1] - poff[v] > kCfWide) continue;  // cf_update_wide_kernel's
    float g[8], x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = 0.0f;
    for (int64_t p = poff[v]; p < poff[v + 1]; ++p) {
      const float4* s = reinterpret_cast<const float4*>(gpart + p * K + d0);
      const float4 a = __ldcs(s), b = __ldcs(s + 1);
      g[0] += a.x; g[1] += a.y; g[2] += a.z; g[3] += a.w;
      g[4] += b.x; g[5] += b.y; g[6] += b.z; g[7] += b.w;
    }
    const int64_t deg = off[v + 1] - off[v];
    const float inv = deg > 0 ? 1.0f / (float)deg : 0.0f;
    load8<PREC>(x0, v, K, d0, x);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = x[q] + step * (g[q] * inv - lambda * x[q]);
    store8<PREC>(x0, v, K, d0, x);
  }
}

// Vertices with more than kCfWide pieces (hub items): one block each.  The
// block's groups of LANES lanes sum interleaved subsets of the pieces (four
// independent accumulators per group, combined in a fixed order), then a
// fixed-order tree over the groups gives the gradient sum; deterministic.
template <int LANES, int PREC>
__global__ void __launch_bounds__(kCfThreads)
cf_update_wide_kernel(const int32_t* __restrict__ wide, int32_t nwide,
                      const int64_t* __restrict__ poff, const int64_t* __restrict__ off,
                      const float* __restrict__ gpart, void* x0, float lambda,
                      float step) {
  constexpr int K = 8 * LANES;
  constexpr int GROUPS = kCfThreads / LANES;
  constexpr int U = 4;
  __shared__ __align__(16) float red[GROUPS * K];
  const int sub = threadIdx.x % LANES, g = threadIdx.x / LANES;
  const int d0 = 8 * sub;
  for (int32_t wv = blockIdx.x; wv < nwide; wv += gridDim.x) {
    const int32_t v = wide[wv];
    const int64_t p0 = poff[v], p1 = poff[v + 1];
    float a[U][8];
#pragma unroll
    for (int j = 0; j < U; ++j)
#pragma unroll
      for (int q = 0; q < 8; ++q) a[j][q] = 0.0f;
    for (int64_t p = p0 + g; p < p1; p += U * GROUPS) {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int64_t pj = p + (int64_t)j * GROUPS;
        if (pj < p1) {
          const float4* s = reinterpret_cast<const float4*>(gpart + pj * K + d0);
          const float4 x = __ldcs(s), y = __ldcs(s + 1);
          a[j][0] += x.x; a[j][1] += x.y; a[j][2] += x.z; a[j][3] += x.w;
          a[j][4] += y.x; a[j][5] += y.y; a[j][6] += y.z; a[j][7] += y.w;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) red[g * K + d0 + q] = (a[0][q] + a[1][q]) + (a[2][q] + a[3][q]);
    __syncthreads();
    for (int st = GROUPS / 2; st >= 1; st >>= 1) {
      if (g < st)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[g * K + d0 + q] += red[(g + st) * K + d0 + q];
      __syncthreads();
    }
    if (g == 0) {
      const int64_t deg = off[v + 1] - off[v];
      const float inv = 1.0f / (float)deg;
      float x[8];
      load8<PREC>(x0, v, K, d0, x);
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = x[q] + step * (red[d0 + q] * inv - lambda * x[q]);
      store8<PREC>(x0, v, K, d0, x);
    }
    __syncthreads();
  }
}

template <int LANES, int PREC>
__global__ void cf_encode_kernel(const float* __restrict__ in, int64_t n, void* x0) {
  constexpr int K = 8 * LANES;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * LANES;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / LANES;
    const int d0 = 8 * (int)(t % LANES);
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = in[v * K + d0 + q];
    store8<PREC>(x0, v, K, d0, x);
  }
}

template <int LANES, int PREC>
__global__ void cf_decode_kernel(const void* x0, int64_t n,
                                 float* __restrict__ out) {
  constexpr int K = 8 * LANES;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * LANES;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / LANES;
    const int d0 = 8 * (int)(t % LANES);
    float x[8];
    load8<PREC>(x0, v, K, d0, x);
#pragma unroll
    for (int q = 0; q < 8; ++q) out[v * K + d0 + q] = x[q];
  }
}

// pieces of each vertex: count, then (after a scan) fill
__global__ void piece_count_kernel(const int64_t* __restrict__ off, int64_t n,
                                   int64_t* __restrict__ cnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    cnt[v] = (off[v + 1] - off[v] + kCfPiece - 1) / kCfPiece;
}

__global__ void piece_fill_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ poff,
                                  int64_t n, int32_t* __restrict__ pvtx,
                                  int64_t* __restrict__ pbeg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = off[v];
    for (int64_t p = poff[v]; p < poff[v + 1]; ++p, b += kCfPiece) {
      pvtx[p] = (int32_t)v;
      pbeg[p] = b;
    }
  }
}

// user of every rating of the user-major CSR, and the item keys to sort by
__global__ void expand_users_kernel(const int64_t* __restrict__ uoff, int64_t U,
                                    const int32_t* __restrict__ uitem, int32_t* __restrict__ user,
                                    uint32_t* __restrict__ key, int32_t* __restrict__ idx) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < U; u += nw)
    for (int64_t e = uoff[u] + lane; e < uoff[u + 1]; e += 32) {
      user[e] = (int32_t)u;
      key[e] = (uint32_t)uitem[e];
      idx[e] = (int32_t)e;
    }
}

__global__ void item_hist_kernel(const int32_t* __restrict__ uitem, int64_t R, int64_t I,
                                 int64_t* __restrict__ cnt, int32_t* __restrict__ bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = uitem[e];
    if (i < 0 || i >= I) {
      atomicExch(bad, 1);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt + i), 1ull);
  }
}

__global__ void transpose_gather_kernel(const int32_t* __restrict__ order, int64_t R,
                                        const int32_t* __restrict__ user,
                                        const uint8_t* __restrict__ urate,
                                        int32_t* __restrict__ iuser, uint8_t* __restrict__ irate) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = order[e];
    iuser[e] = user[s];
    irate[e] = urate[s];
  }
}

template <int LANES, int PREC>
int sweep_side(cg_bipartite* h, int side, double* sse, float lambda, float step, cudaStream_t s,
               bool gather) {
  // side 0: users gather item rows; side 1: items gather user rows
  const int64_t* off = side == 0 ? h->uoff : h->ioff;
  const int32_t* nb = side == 0 ? h->uitem : h->iuser;
  const uint8_t* rt = side == 0 ? h->urate : h->irate;
  void** self = side == 0 ? h->P : h->Q;
  void** other = side == 0 ? h->Q : h->P;
  const int64_t n = side == 0 ? h->U : h->I;
  if (gather) {
    if (h->npieces[side] == 0) {
      if (side == 0 && sse) CG_CUDA(cudaMemsetAsync(sse, 0, sizeof(double), s));
      return CG_OK;
    }
    if (side == 0)
      cf_gather_kernel<LANES, PREC, true><<<h->gather_grid, kCfThreads, 0, s>>>(
          h->pvtx[0], h->pbeg[0], off, h->npieces[0], nb, rt, self[0], other[0], h->gpart[0],
          h->partials, h->counter, sse);
    else
      cf_gather_kernel<LANES, PREC, false><<<h->gather_grid, kCfThreads, 0, s>>>(
          h->pvtx[1], h->pbeg[1], off, h->npieces[1], nb, rt, self[0], other[0], h->gpart[1],
          h->partials, h->counter, nullptr);
  } else {
    cf_update_kernel<LANES, PREC><<<grid_for(n * LANES, kCfThreads, 8), kCfThreads, 0, s>>>(
        h->poff[side], off, n, h->gpart[side], self[0], lambda, step);
    if (h->nwide[side] > 0) {
      CG_LAUNCH_CHECK();
      cf_update_wide_kernel<LANES, PREC><<<h->nwide[side], kCfThreads, 0, s>>>(
          h->wide[side], h->nwide[side], h->poff[side], off, h->gpart[side], self[0],
          lambda, step);
    }
  }
  CG_LAUNCH_CHECK();
  return CG_OK;
}

template <int LANES>
int sweep_dispatch(cg_bipartite* h, int phase, double* sse, float lambda, float step,
                   cudaStream_t s) {
  // phase: 0 user gather, 1 item gather, 2 user update, 3 item update
  const int side = phase & 1;
  const bool gather = phase < 2;
  switch (h->precision) {
    case 0: return sweep_side<LANES, 0>(h, side, sse, lambda, step, s, gather);
    case 1: return sweep_side<LANES, 1>(h, side, sse, lambda, step, s, gather);
    default: return sweep_side<LANES, 2>(h, side, sse, lambda, step, s, gather);
  }
}

int run_phase(cg_bipartite* h, int phase, double* sse, float lambda, float step, cudaStream_t s) {
  switch (h->K) {
    case 16: return sweep_dispatch<2>(h, phase, sse, lambda, step, s);
    case 32: return sweep_dispatch<4>(h, phase, sse, lambda, step, s);
    default: return sweep_dispatch<8>(h, phase, sse, lambda, step, s);
  }
}

template <int LANES>
int codec(cg_bipartite* h, const float* P, const float* Q, float* Pout, float* Qout,
          cudaStream_t s) {
  const int64_t n[2] = {h->U, h->I};
  void** st[2] = {h->P, h->Q};
  const float* in[2] = {P, Q};
  float* out[2] = {Pout, Qout};
  for (int side = 0; side < 2; ++side) {
    if (n[side] == 0) continue;
    const int grid = grid_for(n[side] * LANES, 256, 8);
    if (in[side]) {
      switch (h->precision) {
        case 0: cf_encode_kernel<LANES, 0><<<grid, 256, 0, s>>>(in[side], n[side], st[side][0]); break;
        case 1: cf_encode_kernel<LANES, 1><<<grid, 256, 0, s>>>(in[side], n[side], st[side][0]); break;
        default: cf_encode_kernel<LANES, 2><<<grid, 256, 0, s>>>(in[side], n[side], st[side][0]);
      }
    }
    if (out[side]) {
      switch (h->precision) {
        case 0: cf_decode_kernel<LANES, 0><<<grid, 256, 0, s>>>(st[side][0], n[side], out[side]); break;
        case 1: cf_decode_kernel<LANES, 1><<<grid, 256, 0, s>>>(st[side][0], n[side], out[side]); break;
        default: cf_decode_kernel<LANES, 2><<<grid, 256, 0, s>>>(st[side][0], n[side], out[side]);
      }
    }
    CG_LAUNCH_CHECK();
  }
  return CG_OK;
}

int codec_dispatch(cg_bipartite* h, const float* P, const float* Q, float* Pout, float* Qout,
                   cudaStream_t s) {
  switch (h->K) {
    case 16: return codec<2>(h, P, Q, Pout, Qout, s);
    case 32: return codec<4>(h, P, Q, Pout, Qout, s);
    default: return codec<8>(h, P, Q, Pout, Qout, s);
  }
}

void cf_free(cg_bipartite* h) {
  for (int s = 0; s < 2; ++s) {
    cudaFree(h->pvtx[s]);
    cudaFree(h->pbeg[s]);
    cudaFree(h->poff[s]);
    cudaFree(h->gpart[s]);
    cudaFree(h->wide[s]);
    cudaFree(h->P[s]);
    cudaFree(h->Q[s]);
  }
  cudaFree(h->partials);
  cudaFree(h->counter);
  delete h;
}

int build_pieces(cg_bipartite* h, int side, cudaStream_t s) {
  const int64_t* off = side == 0 ? h->uoff : h->ioff;
  const int64_t n = side == 0 ? h->U : h->I;
  int64_t* cnt = nullptr;
  CG_CUDA(cudaMalloc((void**)&h->poff[side], sizeof(int64_t) * (size_t)(n + 1)));
  h->bytes += 8 * (n + 1);
  CG_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int64_t) * (size_t)(n > 0 ? n : 1), s));
  int st = CG_OK;
  if (n > 0) {
    piece_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "piece_count", __FILE__, __LINE__);
    if (st == CG_OK) st = exclusive_scan_i64(cnt, h->poff[side], n, s);
  } else {
    cudaError_t e = cudaMemsetAsync(h->poff[side], 0, sizeof(int64_t), s);
    if (e != cudaSuccess) st = cuda_fail(e, "poff", __FILE__, __LINE__);
  }
  cudaFreeAsync(cnt, s);
  if (st != CG_OK) return st;
  int64_t np = 0;
  CG_CUDA(cudaMemcpyAsync(&np, h->poff[side] + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  h->npieces[side] = np;
  const size_t m = (size_t)(np > 0 ? np : 1);
  CG_CUDA(cudaMalloc((void**)&h->pvtx[side], sizeof(int32_t) * m));
  CG_CUDA(cudaMalloc((void**)&h->pbeg[side], sizeof(int64_t) * m));
  CG_CUDA(cudaMalloc((void**)&h->gpart[side], sizeof(float) * m * h->K));
  CG_CUDA(cudaMemsetAsync(h->gpart[side], 0, sizeof(float) * m * h->K, s));
  h->bytes += (int64_t)m * (12 + 4 * h->K);
  if (n > 0 && np > 0) {
    piece_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, h->poff[side], n, h->pvtx[side],
                                                        h->pbeg[side]);
    CG_LAUNCH_CHECK();
  }
  // vertices with many pieces get a whole block in the update
  std::vector<int64_t> hp((size_t)n + 1);
  CG_CUDA(cudaMemcpyAsync(hp.data(), h->poff[side], sizeof(int64_t) * (size_t)(n + 1),
                          cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> wide;
  for (int64_t v = 0; v < n; ++v)
    if (hp[v + 1] - hp[v] > kCfWide) wide.push_back((int32_t)v);
  h->nwide[side] = (int32_t)wide.size();
  if (!wide.empty()) {
    CG_CUDA(cudaMalloc((void**)&h->wide[side], sizeof(int32_t) * wide.size()));
    h->bytes += 4 * (int64_t)wide.size();
    CG_CUDA(cudaMemcpyAsync(h->wide[side], wide.data(), sizeof(int32_t) * wide.size(),
                            cudaMemcpyHostToDevice, s));
    CG_CUDA(cudaStreamSynchronize(s));
  }
  return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int cf_transpose(int64_t U, int64_t I, const int64_t* uoff, const int32_t* uitem,
                 const uint8_t* urate, int64_t* ioff, int32_t* iuser, uint8_t* irate,
                 cudaStream_t stream) {
  CG_ARG(U >= 0 && I >= 1 && I < (int64_t)1 << 31, "cf_transpose: need U >= 0, 1 <= I < 2^31");
  CG_ARG(uoff && ioff, "cf_transpose: null offsets");
  int64_t R = 0;
  CG_CUDA(cudaMemcpyAsync(&R, uoff + U, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  CG_CUDA(cudaStreamSynchronize(stream));
  CG_ARG(R >= 0 && R < 0x7FFFFFFFLL, "cf_transpose: rating count %lld out of range",
         (long long)R);
  CG_ARG(R == 0 || (uitem && urate && iuser && irate), "cf_transpose: null rating arrays");
  int64_t* cnt = nullptr;
  int32_t *user = nullptr, *idx = nullptr, *order = nullptr, *bad = nullptr;
  uint32_t *key = nullptr, *key2 = nullptr;
  const size_t Rm = (size_t)(R > 0 ? R : 1);
  cudaError_t e = cudaMallocAsync((void**)&cnt, sizeof(int64_t) * (size_t)I, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&bad, sizeof(int32_t), stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&user, sizeof(int32_t) * Rm, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&idx, sizeof(int32_t) * Rm, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&order, sizeof(int32_t) * Rm, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&key, sizeof(uint32_t) * Rm, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&key2, sizeof(uint32_t) * Rm, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)I, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int32_t), stream);
  int st = CG_OK;
  if (e == cudaSuccess && R > 0) {
    item_hist_kernel<<<grid_for(R, 256), 256, 0, stream>>>(uitem, R, I, cnt, bad);
    e = cudaGetLastError();
  }
  int32_t hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                            stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess && hbad) {
    set_error("cf_transpose: an item index is outside [0, %lld)", (long long)I);
    st = CG_ERR_INVALID_ARG;
  }
  if (e == cudaSuccess && st == CG_OK) st = exclusive_scan_i64(cnt, ioff, I, stream);
  if (e == cudaSuccess && st == CG_OK && R > 0) {
    expand_users_kernel<<<grid_for(U * 32, 256), 256, 0, stream>>>(uoff, U, uitem, user, key,
                                                                    idx);
    e = cudaGetLastError();
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < I) ++bits;
    // stable sort by item: users stay ascending within each item
    if (e == cudaSuccess) st = radix_sort_pairs(key, idx, key2, order, R, bits, stream);
    if (e == cudaSuccess && st == CG_OK) {
      transpose_gather_kernel<<<grid_for(R, 256), 256, 0, stream>>>(order, R, user, urate, iuser,
                                                                    irate);
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(cnt, stream);
  cudaFreeAsync(bad, stream);
  cudaFreeAsync(user, stream);
  cudaFreeAsync(idx, stream);
  cudaFreeAsync(order, stream);
  cudaFreeAsync(key, stream);
  cudaFreeAsync(key2, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cf_transpose", __FILE__, __LINE__);
  return st;
}

int cf_create(int64_t U, int64_t I, int32_t K, int32_t precision, const int64_t* uoff,
              const int32_t* uitem, const uint8_t* urate, const int64_t* ioff,
              const int32_t* iuser, const uint8_t* irate, cg_bipartite** out,
              cudaStream_t stream) {
  CG_ARG(out != nullptr, "cf_create: out is NULL");
  *out = nullptr;
  CG_ARG(U >= 1 && I >= 1 && U < (int64_t)1 << 31 && I < (int64_t)1 << 31,
         "cf_create: need 1 <= U, I < 2^31");
  CG_ARG(K == 16 || K == 32 || K == 64, "cf_create: K must be 16, 32 or 64 (got %d)", K);
  CG_ARG(precision >= 0 && precision <= 2,
         "cf_create: precision must be 0 (FP32), 1 (BF16) or 2 (BF16 hi+lo), got %d", precision);
  CG_ARG(uoff && ioff, "cf_create: null offsets");
  int64_t R = 0, R2 = 0;
  CG_CUDA(cudaMemcpyAsync(&R, uoff + U, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  CG_CUDA(cudaMemcpyAsync(&R2, ioff + I, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  CG_CUDA(cudaStreamSynchronize(stream));
  CG_ARG(R == R2 && R >= 0, "cf_create: user side has %lld ratings, item side %lld",
         (long long)R, (long long)R2);
  CG_ARG(R == 0 || (uitem && urate && iuser && irate), "cf_create: null rating arrays");
  cg_bipartite* h = new cg_bipartite();
  CG_CUDA(cudaGetDevice(&h->device));
  h->U = U;
  h->I = I;
  h->R = R;
  h->K = K;
  h->precision = precision;
  h->uoff = uoff;
  h->uitem = uitem;
  h->urate = urate;
  h->ioff = ioff;
  h->iuser = iuser;
  h->irate = irate;
  int st = build_pieces(h, 0, stream);
  if (st == CG_OK) st = build_pieces(h, 1, stream);
  cudaError_t e = cudaSuccess;
  const size_t el = precision == 1 ? 2 : 4;  // BF16 hi + lo: one 32-bit word per entry
  const int planes = 1;
  for (int pl = 0; pl < planes && st == CG_OK && e == cudaSuccess; ++pl) {
    e = cudaMalloc(&h->P[pl], el * (size_t)U * K);
    if (e == cudaSuccess) e = cudaMalloc(&h->Q[pl], el * (size_t)I * K);
    h->bytes += (int64_t)(el * (size_t)(U + I) * K);
  }
  if (st == CG_OK && e == cudaSuccess) {
    DeviceInfo di{};
    st = device_info(&di);
    h->gather_grid = di.sm_count * 8;  // 2048 threads per SM at 256 per block
    if (st == CG_OK) e = cudaMalloc((void**)&h->partials, sizeof(double) * h->gather_grid);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->counter, 0, sizeof(unsigned), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  }
  if (st == CG_OK && e != cudaSuccess) st = cuda_fail(e, "cf_create", __FILE__, __LINE__);
  if (st != CG_OK) {
    cudaStreamSynchronize(stream);
    cf_free(h);
    return st;
  }
  *out = h;
  return CG_OK;
}

int cf_destroy(cg_bipartite* h) {
  if (!h) return CG_OK;
  cudaDeviceSynchronize();
  cf_free(h);
  return CG_OK;
}

int cf_set_factors(cg_bipartite* h, const float* P, const float* Q, cudaStream_t stream) {
  CG_ARG(h && P && Q, "cf_set_factors: null argument");
  return codec_dispatch(h, P, Q, nullptr, nullptr, stream);
}

int cf_get_factors(const cg_bipartite* h, float* P, float* Q, cudaStream_t stream) {
  CG_ARG(h, "cf_get_factors: null handle");
  return codec_dispatch(const_cast<cg_bipartite*>(h), nullptr, nullptr, P, Q, stream);
}

int cf_sweep(cg_bipartite* h, int32_t sweeps, double lambda, double step, double* sse,
             cudaStream_t stream) {
  CG_ARG(h, "cf_sweep: null handle");
  CG_ARG(sweeps >= 1, "cf_sweep: sweeps must be >= 1");
  CG_ARG(lambda >= 0.0 && step >= 0.0, "cf_sweep: lambda and step must be >= 0");
  for (int t = 0; t < sweeps; ++t)
    for (int phase = 0; phase < 4; ++phase)
      CG_TRY(run_phase(h, phase, sse ? sse + t : nullptr, (float)lambda, (float)step, stream));
  return CG_OK;
}

int cf_sweep_phase(cg_bipartite* h, int32_t phase, double lambda, double step, double* sse,
                   cudaStream_t stream) {
  CG_ARG(h, "cf_sweep_phase: null handle");
  CG_ARG(phase >= 0 && phase <= 3, "cf_sweep_phase: phase must be in [0, 3]");
  return run_phase(h, phase, sse, (float)lambda, (float)step, stream);
}

int cf_info(const cg_bipartite* h, int64_t* ratings, int64_t* user_pieces, int64_t* item_pieces,
            int64_t* bytes) {
  CG_ARG(h, "cf_info: null handle");
  if (ratings) *ratings = h->R;
  if (user_pieces) *user_pieces = h->npieces[0];
  if (item_pieces) *item_pieces = h->npieces[1];
  if (bytes) *bytes = h->bytes;
  return CG_OK;
}

}  // extern "C"
