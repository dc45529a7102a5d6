// Batched PageRank over many small graphs in one persistent launch.
//
// Each graph is small enough that its whole contrib vector fits in one SM's
// shared memory, so a graph is its own single shared-memory segment (k = 1
// in the paper's terms) and a block runs all of its iterations on chip:
//   gather   warps take 256-edge chunks of the graph's flagged edge stream
//            (bit 31 = last edge of a destination row) and fold contrib from
//            shared memory, exactly as the segment gather does;
//   carries  rows spanning chunks are completed in chunk order;
//   merge    the non-empty rows' sums are scattered into a dense shared
//            accumulator (k = 1: one row per destination, no collisions);
//   update   the normalised vertex update, the FP64 dangling mass and the L1
//            residual, and the next contrib written back into shared memory.
// Graphs are handed out largest first through an atomic counter, so the
// biggest ones start first and small ones fill in behind (longest processing
// time first).  Nothing waits on another block.
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "gather.cuh"

struct cg_batch {
  int device = 0;
  int32_t G = 0;
  int64_t V = 0, E = 0, rows = 0, nchunks = 0;
  int32_t vmax = 0;
  std::vector<int64_t> h_vbase, h_ebase;
  // per graph (device): vertex / edge / non-empty-row / chunk bases, dangling count
  int64_t* vbase = nullptr;   // [G+1]
  int64_t* ebase = nullptr;   // [G+1]
  int64_t* rbase = nullptr;   // [G+1]
  int64_t* cbase = nullptr;   // [G+1]
  int32_t* order = nullptr;   // [G] graphs by edge count, descending
  int32_t* ndang = nullptr;   // [G]
  uint32_t* colf = nullptr;   // [E + 256] local source | row-end flag
  int32_t* idx = nullptr;     // [rows] local destination of each non-empty row
  int32_t* first_row = nullptr;  // [nchunks] graph-local non-empty row of each chunk's first edge
  float* inv = nullptr;       // [V]
  float* interm = nullptr;    // [rows]
  float* carry = nullptr;     // [nchunks]
  int32_t* carry_row = nullptr;  // [nchunks]
  unsigned* counter = nullptr;
  int threads = 1024;
  int64_t bytes = 0;
};

namespace cg {
namespace {

constexpr int kBatchChunk = 256;

__global__ void batch_degree_kernel(const int32_t* __restrict__ src, const int64_t* __restrict__ ebase,
                                    const int64_t* __restrict__ vbase, int G, int64_t E,
                                    int32_t* __restrict__ outdeg) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = G + 1;  // graph of edge e: last g with ebase[g] <= e
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ebase[mid] <= e) lo = mid + 1; else hi = mid;
    }
    const int g = lo - 1;
    const int32_t u = src[e];
    if (u >= 0 && (int64_t)u < vbase[g + 1] - vbase[g]) atomicAdd(outdeg + vbase[g] + u, 1);
  }
}

__global__ void batch_inv_kernel(const int32_t* __restrict__ outdeg, int64_t V,
                                 float* __restrict__ inv, const int64_t* __restrict__ offsets,
                                 int32_t* __restrict__ nonempty) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    inv[v] = outdeg[v] > 0 ? 1.0f / (float)outdeg[v] : 0.0f;
    nonempty[v] = offsets[v + 1] > offsets[v] ? 1 : 0;
  }
}

// Flagged edges and the non-empty row index (rows in vertex order).
__global__ void batch_rows_kernel(const int64_t* __restrict__ offsets,
                                  const int32_t* __restrict__ src,
                                  const int64_t* __restrict__ rowpos,  // exclusive scan of nonempty
                                  const int64_t* __restrict__ vbase, int G, int64_t V,
                                  uint32_t* __restrict__ colf, int32_t* __restrict__ idx) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nw) {
    const int64_t lo = offsets[v], hi = offsets[v + 1];
    if (hi == lo) continue;
    if (lane == 0) {
      int a = 0, b = G + 1;
      while (a < b) {
        const int mid = (a + b) >> 1;
        if (vbase[mid] <= v) a = mid + 1; else b = mid;
      }
      idx[rowpos[v]] = (int32_t)(v - vbase[a - 1]);
    }
    for (int64_t e = lo + lane; e < hi; e += 32)
      colf[e] = (uint32_t)src[e] | (e == hi - 1 ? 0x80000000u : 0u);
  }
}

// Graph-local non-empty row of each chunk's first edge; also the dangling
// count per graph is accumulated here by a separate kernel.
__global__ void batch_first_row_kernel(const int64_t* __restrict__ offsets,
                                       const int64_t* __restrict__ rowpos,
                                       const int64_t* __restrict__ vbase,
                                       const int64_t* __restrict__ ebase,
                                       const int64_t* __restrict__ rbase,
                                       const int64_t* __restrict__ cbase, int G,
                                       int64_t nchunks, int32_t* __restrict__ first_row) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    int a = 0, b = G + 1;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (cbase[mid] <= c) a = mid + 1; else b = mid;
    }
    const int g = a - 1;
    const int64_t e = ebase[g] + (c - cbase[g]) * kBatchChunk;
    // vertex whose row holds edge e: last v in the graph with offsets[v] <= e (non-empty)
    int64_t lo = vbase[g], hi = vbase[g + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (offsets[mid] <= e) lo = mid + 1; else hi = mid;
    }
    first_row[c] = (int32_t)(rowpos[lo - 1] - rbase[g]);
  }
}

__global__ void batch_dangling_kernel(const int32_t* __restrict__ outdeg,
                                      const int64_t* __restrict__ vbase, int G,
                                      int32_t* __restrict__ ndang) {
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    int c = 0;
    for (int64_t v = vbase[g] + threadIdx.x; v < vbase[g + 1]; v += blockDim.x)
      c += outdeg[v] == 0;
    c = warp_sum(c);
    __shared__ int sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
      ndang[g] = t;
    }
    __syncthreads();
  }
}

struct BatchArgs {
  const uint32_t* colf;
  const int32_t* idx;
  const int32_t* first_row;
  const float* inv;
  const int64_t *vbase, *ebase, *rbase, *cbase;
  const int32_t* order;
  const int32_t* ndang;
  float* interm;
  float* carry;
  int32_t* carry_row;
  float* rank;     // [V] result (and the previous iterate while running)
  double* resid;   // [G * iters] or NULL
  unsigned* counter;
  int G;
  int iters;
  float d;
};

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
batch_pagerank_kernel(BatchArgs a) {
  constexpr int WARPS = THREADS / 32;
  extern __shared__ __align__(16) float xs[];  // contrib, then the gathered sums
  __shared__ int s_g;
  __shared__ double s_red[2][WARPS];
  __shared__ double s_D;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const unsigned q = atomicAdd(a.counter, 1u);
      s_g = (int)q < a.G ? a.order[q] : -1;
    }
    __syncthreads();
    const int g = s_g;
    if (g < 0) break;
    const int64_t vb = a.vbase[g], eb = a.ebase[g], rb = a.rbase[g], cb = a.cbase[g];
    const int V = (int)(a.vbase[g + 1] - vb);
    const int E = (int)(a.ebase[g + 1] - eb);
    const int nch = (int)(a.cbase[g + 1] - cb);
    const float base = (1.0f - a.d) / (float)V;
    const double invV = 1.0 / (double)V;
    float* rank = a.rank + vb;
    const float* inv = a.inv + vb;
    // r_0 = 1/V
    const float r0 = 1.0f / (float)V;
    for (int v = tid; v < V; v += THREADS) {
      rank[v] = r0;
      xs[v] = r0 * inv[v];
    }
    double D = (double)a.ndang[g] * (double)r0;
    __syncthreads();
    for (int it = 0; it < a.iters; ++it) {
      // 1. gather: flagged 256-edge chunks, sources from shared memory
      for (int j = w; j < nch; j += WARPS) {
        const int e0 = j * kBatchChunk;
        const int n = E - e0 < kBatchChunk ? E - e0 : kBatchChunk;
        const int64_t c = cb + j;
        const int32_t frow = a.first_row[c];
        const uint4* p = reinterpret_cast<const uint4*>(a.colf + eb + e0 + lane * 8);
        uint32_t cf[8];
        if (((eb + e0) & 3) == 0) {  // 16-byte aligned chunk
          const uint4 qa = __ldg(p), qb = __ldg(p + 1);
          cf[0] = qa.x; cf[1] = qa.y; cf[2] = qa.z; cf[3] = qa.w;
          cf[4] = qb.x; cf[5] = qb.y; cf[6] = qb.z; cf[7] = qb.w;
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u) cf[u] = __ldg(a.colf + eb + e0 + lane * 8 + u);
        }
        float v[8];
        uint32_t fl = 0;
        const int nl = n - lane * 8;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool ok = u < nl;
          const uint32_t s = cf[u] & 0x7FFFFFFFu;
          if (ok) fl |= (cf[u] >> 31) << u;
          v[u] = (ok && s < (uint32_t)V) ? xs[s] : 0.0f;
        }
        const int F = __popc(fl);
        int incl = F;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int32_t row0 = frow + (incl - F);
        float acc = 0.0f, first_val = 0.0f;
        int nf = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc += v[u];
          if (fl & (1u << u)) {
            if (nf == 0) first_val = acc;
            else a.interm[rb + row0 + nf] = acc;
            ++nf;
            acc = 0.0f;
          }
        }
        float S = acc;
        int h = F > 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float y = __shfl_up_sync(0xffffffffu, S, o);
          const int gg = __shfl_up_sync(0xffffffffu, h, o);
          if (lane >= o) {
            if (!h) S = y + S;
            h |= gg;
          }
        }
        const float P = __shfl_up_sync(0xffffffffu, S, 1);
        if (F > 0) a.interm[rb + row0] = lane > 0 ? P + first_val : first_val;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t lf = __shfl_sync(0xffffffffu, fl, (n - 1) >> 3);
        if (lane == 31) {
          const bool closed = (lf >> ((n - 1) & 7)) & 1u;
          a.carry[c] = closed ? 0.0f : S;
          a.carry_row[c] = closed ? -1 : frow + total;
        }
      }
      __syncthreads();
      // 2. rows spanning chunks: the first chunk of each run sums the run
      for (int j = tid; j < nch; j += THREADS) {
        const int32_t r = a.carry_row[cb + j];
        if (r < 0 || (j > 0 && a.carry_row[cb + j - 1] == r)) continue;
        float s = a.carry[cb + j];
        for (int u = j + 1; u < nch && a.carry_row[cb + u] == r; ++u) s += a.carry[cb + u];
        a.interm[rb + r] += s;
      }
      __syncthreads();
      // 3. merge into a dense accumulator (k = 1: one row per destination)
      for (int v = tid; v < V; v += THREADS) xs[v] = 0.0f;
      __syncthreads();
      const int nrows = (int)(a.rbase[g + 1] - rb);
      for (int r0 = tid; r0 < nrows; r0 += THREADS * 4) {  // four rows' loads in flight
        int32_t dv[4];
        float val[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = r0 + u * THREADS;
          dv[u] = r < nrows ? a.idx[rb + r] : -1;
          val[u] = r < nrows ? a.interm[rb + r] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((uint32_t)dv[u] < (uint32_t)V) xs[dv[u]] = val[u];
      }
      __syncthreads();
      // 4. vertex update, next contrib, FP64 dangling mass and residual
      const float Dv = (float)(D * invV);
      float dpart = 0.0f, rpart = 0.0f;
      constexpr int U = 8;  // vertices per thread whose inputs are loaded together
      for (int v0 = tid; v0 < V; v0 += THREADS * U) {
        float iv[U], old[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int v = v0 + u * THREADS;
          iv[u] = v < V ? inv[v] : 0.0f;
          old[u] = v < V ? rank[v] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {  // the same vertex order as one at a time
          const int v = v0 + u * THREADS;
          if (v < V) {
            const float r = base + a.d * (xs[v] + Dv);
            rpart += fabsf(r - old[u]);
            rank[v] = r;
            xs[v] = r * iv[u];
            if (iv[u] == 0.0f) dpart += r;
          }
        }
      }
      // the lanes' partials in FP32 over groups of 2o lanes while a group
      // holds at most 256 ranks (ceil(V / THREADS) per lane), then in FP64
      const int per_lane = (V + THREADS - 1) / THREADS;
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
      if (lane == 0) {
        s_red[0][w] = dd;
        s_red[1][w] = rr;
      }
      __syncthreads();
      // one thread adds the warps' sums in warp order (FP64 runs at a small
      // fraction of the FP32 rate on this GPU: every thread repeating the loop
      // cost more than the rest of the update) and shares the result
      if (tid == 0) {
        double Dn = 0.0, Rn = 0.0;
        for (int q = 0; q < WARPS; ++q) {
          Dn += s_red[0][q];
          Rn += s_red[1][q];
        }
        s_D = Dn;
        if (a.resid) a.resid[(int64_t)g * a.iters + it] = Rn;
      }
      __syncthreads();
      D = s_D;
    }
  }
}

void free_batch(cg_batch* b) {
  cudaFree(b->vbase);
  cudaFree(b->ebase);
  cudaFree(b->rbase);
  cudaFree(b->cbase);
  cudaFree(b->order);
  cudaFree(b->ndang);
  cudaFree(b->colf);
  cudaFree(b->idx);
  cudaFree(b->first_row);
  cudaFree(b->inv);
  cudaFree(b->interm);
  cudaFree(b->carry);
  cudaFree(b->carry_row);
  cudaFree(b->counter);
}

int build_batch(cg_batch* b, const int64_t* offsets, const int32_t* src, cudaStream_t s) {
  const int G = b->G;
  // per-graph edge bases from the offsets (host reads G+1 values)
  b->h_ebase.assign(G + 1, 0);
  for (int g = 0; g <= G; ++g)
    CG_CUDA(cudaMemcpyAsync(&b->h_ebase[g], offsets + b->h_vbase[g], sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  if (b->h_ebase[0] != 0) {
    set_error("pr_batch_create: offsets must start at 0");
    return CG_ERR_INVALID_ARG;
  }
  for (int g = 0; g < G; ++g)
    if (b->h_ebase[g + 1] < b->h_ebase[g]) {
      set_error("pr_batch_create: offsets decrease across graph %d", g);
      return CG_ERR_INVALID_ARG;
    }
  b->E = b->h_ebase[G];
  std::vector<int64_t> cbase(G + 1, 0);
  for (int g = 0; g < G; ++g)
    cbase[g + 1] = cbase[g] + ceil_div(b->h_ebase[g + 1] - b->h_ebase[g], kBatchChunk);
  b->nchunks = cbase[G];
  std::vector<int32_t> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->h_ebase[x + 1] - b->h_ebase[x] > b->h_ebase[y + 1] - b->h_ebase[y];
  });
  const int64_t V = b->V, E = b->E;
  CG_CUDA(cudaMalloc((void**)&b->vbase, sizeof(int64_t) * (G + 1)));
  CG_CUDA(cudaMalloc((void**)&b->ebase, sizeof(int64_t) * (G + 1)));
  CG_CUDA(cudaMalloc((void**)&b->rbase, sizeof(int64_t) * (G + 1)));
  CG_CUDA(cudaMalloc((void**)&b->cbase, sizeof(int64_t) * (G + 1)));
  CG_CUDA(cudaMalloc((void**)&b->order, sizeof(int32_t) * G));
  CG_CUDA(cudaMalloc((void**)&b->ndang, sizeof(int32_t) * G));
  CG_CUDA(cudaMalloc((void**)&b->colf, sizeof(uint32_t) * (size_t)(E + kBatchChunk)));
  CG_CUDA(cudaMalloc((void**)&b->inv, sizeof(float) * (size_t)V));
  CG_CUDA(cudaMalloc((void**)&b->first_row, sizeof(int32_t) * (size_t)(b->nchunks + 1)));
  CG_CUDA(cudaMalloc((void**)&b->carry, sizeof(float) * (size_t)(b->nchunks + 1)));
  CG_CUDA(cudaMalloc((void**)&b->carry_row, sizeof(int32_t) * (size_t)(b->nchunks + 1)));
  CG_CUDA(cudaMalloc((void**)&b->counter, sizeof(unsigned)));
  CG_CUDA(cudaMemsetAsync(b->colf, 0, sizeof(uint32_t) * (size_t)(E + kBatchChunk), s));
  CG_CUDA(cudaMemcpyAsync(b->vbase, b->h_vbase.data(), sizeof(int64_t) * (G + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(b->ebase, b->h_ebase.data(), sizeof(int64_t) * (G + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(b->cbase, cbase.data(), sizeof(int64_t) * (G + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(b->order, order.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s));
  // scratch: out-degree, non-empty flags and their scan
  int32_t *outdeg = nullptr, *nonempty = nullptr;
  int64_t* rowpos = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&outdeg, sizeof(int32_t) * (size_t)V, s));
  CG_CUDA(cudaMallocAsync((void**)&nonempty, sizeof(int32_t) * (size_t)V, s));
  CG_CUDA(cudaMallocAsync((void**)&rowpos, sizeof(int64_t) * (size_t)(V + 1), s));
  int st = CG_OK;
  cudaError_t e = cudaMemsetAsync(outdeg, 0, sizeof(int32_t) * (size_t)V, s);
  if (e == cudaSuccess && E > 0) {
    batch_degree_kernel<<<grid_for(E, 256), 256, 0, s>>>(src, b->ebase, b->vbase, G, E, outdeg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    batch_inv_kernel<<<grid_for(V, 256), 256, 0, s>>>(outdeg, V, b->inv, offsets, nonempty);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    batch_dangling_kernel<<<std::min(G, 4096), 256, 0, s>>>(outdeg, b->vbase, G, b->ndang);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) st = cuda_fail(e, "pr_batch_create", __FILE__, __LINE__);
  if (st == CG_OK) st = exclusive_scan_i32_to_i64(nonempty, rowpos, V, s);
  std::vector<int64_t> rbase(G + 1, 0);
  if (st == CG_OK) {
    for (int g = 0; g <= G; ++g) {
      e = cudaMemcpyAsync(&rbase[g], rowpos + b->h_vbase[g], sizeof(int64_t),
                          cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "pr_batch_create rows", __FILE__, __LINE__);
  }
  if (st == CG_OK) {
    b->rows = rbase[G];
    e = cudaMalloc((void**)&b->idx, sizeof(int32_t) * (size_t)(b->rows + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->interm, sizeof(float) * (size_t)(b->rows + 1));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->rbase, rbase.data(), sizeof(int64_t) * (G + 1),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      batch_rows_kernel<<<grid_for(V * 32, 256, 16), 256, 0, s>>>(offsets, src, rowpos, b->vbase,
                                                                  G, V, b->colf, b->idx);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && b->nchunks > 0) {
      batch_first_row_kernel<<<grid_for(b->nchunks, 256), 256, 0, s>>>(
          offsets, rowpos, b->vbase, b->ebase, b->rbase, b->cbase, G, b->nchunks, b->first_row);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "pr_batch_create build", __FILE__, __LINE__);
  }
  cudaFreeAsync(outdeg, s);
  cudaFreeAsync(nonempty, s);
  cudaFreeAsync(rowpos, s);
  cudaStreamSynchronize(s);
  b->bytes = 4 * (E + kBatchChunk) + 4 * V + 8 * (b->rows + 1) + 12 * (b->nchunks + 1) +
             40 * (int64_t)(G + 1);
  return st;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int pr_batch_create(int32_t G, const int64_t* host_vbase, const int64_t* offsets,
                    const int32_t* src, cg_batch** out, cudaStream_t stream) {
  CG_ARG(out != nullptr, "pr_batch_create: out is NULL");
  *out = nullptr;
  CG_ARG(G >= 1 && host_vbase && offsets, "pr_batch_create: bad arguments");
  CG_ARG(host_vbase[0] == 0, "pr_batch_create: vertex bases must start at 0");
  int32_t vmax = 0;
  for (int g = 0; g < G; ++g) {
    const int64_t n = host_vbase[g + 1] - host_vbase[g];
    CG_ARG(n >= 1, "pr_batch_create: graph %d has no vertex", g);
    CG_ARG(n <= 65536, "pr_batch_create: graph %d has %lld vertices (at most 65536: a graph's "
           "contrib must fit in shared memory)", g, (long long)n);
    vmax = std::max<int32_t>(vmax, (int32_t)n);
  }
  cg_batch* b = new cg_batch();
  CG_CUDA(cudaGetDevice(&b->device));
  b->G = G;
  b->V = host_vbase[G];
  b->vmax = vmax;
  b->h_vbase.assign(host_vbase, host_vbase + G + 1);
  const int cap = (int)((232448 - 2048) / 4);  // shared memory of one block, in floats
  if (vmax > cap) {
    delete b;
    set_error("pr_batch_create: largest graph (%d vertices) exceeds shared memory", vmax);
    return CG_ERR_UNSUPPORTED;
  }
  int st = build_batch(b, offsets, src, stream);
  if (st != CG_OK) {
    cudaStreamSynchronize(stream);
    free_batch(b);
    delete b;
    return st;
  }
  *out = b;
  return CG_OK;
}

int pr_batch_destroy(cg_batch* b) {
  if (!b) return CG_OK;
  int cur = 0;
  const int dev = b->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  free_batch(b);
  delete b;
  if (cur != dev) cudaSetDevice(cur);
  return CG_OK;
}

int pr_batch_set_threads(cg_batch* b, int32_t threads) {
  CG_ARG(b != nullptr, "pr_batch_set_threads: null handle");
  CG_ARG(threads == 256 || threads == 512 || threads == 1024,
         "pr_batch_set_threads: threads must be 256, 512 or 1024");
  b->threads = threads;
  return CG_OK;
}

int pr_batch_run(cg_batch* b, int32_t iterations, double damping, float* rank,
                 double* resid, cudaStream_t stream) {
  CG_ARG(b && rank, "pr_batch_run: null argument");
  CG_ARG(iterations >= 1, "pr_batch_run: iterations must be >= 1");
  CG_ARG(damping >= 0.0 && damping <= 1.0, "pr_batch_run: damping must be in [0, 1]");
  BatchArgs a;
  a.colf = b->colf;
  a.idx = b->idx;
  a.first_row = b->first_row;
  a.inv = b->inv;
  a.vbase = b->vbase;
  a.ebase = b->ebase;
  a.rbase = b->rbase;
  a.cbase = b->cbase;
  a.order = b->order;
  a.ndang = b->ndang;
  a.interm = b->interm;
  a.carry = b->carry;
  a.carry_row = b->carry_row;
  a.rank = rank;
  a.resid = resid;
  a.counter = b->counter;
  a.G = b->G;
  a.iters = iterations;
  a.d = (float)damping;
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  const size_t smem = (size_t)b->vmax * sizeof(float);
  const int per_sm = std::max(1, std::min(2048 / b->threads,
                                          (int)(232448 / std::max<size_t>(smem + 2048, 1))));
  const int grid = std::min<int>(b->G, di.sm_count * per_sm);
  CG_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(unsigned), stream));
  const void* fn = b->threads == 1024 ? (const void*)batch_pagerank_kernel<1024>
                   : b->threads == 512 ? (const void*)batch_pagerank_kernel<512>
                                       : (const void*)batch_pagerank_kernel<256>;
  if (smem > 48 * 1024)
    CG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (b->threads == 1024)
    batch_pagerank_kernel<1024><<<grid, 1024, smem, stream>>>(a);
  else if (b->threads == 512)
    batch_pagerank_kernel<512><<<grid, 512, smem, stream>>>(a);
  else
    batch_pagerank_kernel<256><<<grid, 256, smem, stream>>>(a);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int pr_batched_graphs_run(cg_batch* b, int32_t iterations, double damping, float* rank,
                          double* resid, cudaStream_t stream) {
  return pr_batch_run(b, iterations, damping, rank, resid, stream);
}

}  // extern "C"
