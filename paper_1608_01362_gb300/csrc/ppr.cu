// Batched personalised PageRank: 64 rank vectors advanced together over one
// segmented graph.  Each iteration is Algorithm 3's gather and Algorithm 4's
// merge with 64-wide rows in place of scalars (an SpMM with a 64-column dense
// operand), followed by the personalised form of Algorithm 5's update:
//   R'[v][j] = d (sum_{u->v} C[u][j]) + [v == seed_j] ((1-d) + d D_j)
//   C'[v][j] = R'[v][j] / outdeg(v),     D'_j = sum_{outdeg(v)=0} R'[v][j]
// (the teleport and the dangling mass of column j return to its seed).
//
// Storage.  The iteration state is C (the contributions R/outdeg) of the
// non-dangling vertices, as BF16 planes: hi = bf16(c) and, with two planes,
// lo = bf16(c - hi), 128 bytes per vertex per plane.  Gathers read the
// planes and accumulate hi + lo in FP32.  R itself is written in FP32 only
// when asked for (the last iteration, and the one before it for the L1
// residual); D_j and the residual are FP64 with a fixed reduction order.
//
// Kernels per iteration:
//   ppr_gather_kernel  an octet (8 lanes, 8 columns each) walks a 128-edge
//                      chunk of one segment's flagged edge stream, reading
//                      C rows of the segment's sources (a slice sized to
//                      stay in L2), and writes each subgraph row's 64 sums
//                      to intermBuf; the row open at the chunk's end goes
//                      to a carry slot;
//   ppr_fixup_kernel   completes the rows that span chunks: each run of
//                      carries (consecutive chunks open on the same row, a
//                      static structure) is cut into pieces of <= 32 chunks
//                      summed in parallel; the last piece of a run adds the
//                      pieces' sums, in order, into the row;
//   ppr_merge_kernel   an octet takes 16 consecutive destinations, sums
//                      their intermBuf rows (destination-major list of the
//                      rows, in segment order), applies the update and
//                      writes C' (and R'), with per-column FP64 partials
//                      reduced by the last block.
#include "ppr.cuh"

namespace cg {
namespace {

// BF16 pairs (element 0 in the low half) to FP32: exact.
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void add_row(float (&acc)[8], const uint4& h) {
  acc[0] += bf_lo(h.x); acc[1] += bf_hi(h.x);
  acc[2] += bf_lo(h.y); acc[3] += bf_hi(h.y);
  acc[4] += bf_lo(h.z); acc[5] += bf_hi(h.z);
  acc[6] += bf_lo(h.w); acc[7] += bf_hi(h.w);
}

__device__ __forceinline__ void add_row2(float (&acc)[8], const uint4& h, const uint4& l) {
  acc[0] += bf_lo(h.x) + bf_lo(l.x); acc[1] += bf_hi(h.x) + bf_hi(l.x);
  acc[2] += bf_lo(h.y) + bf_lo(l.y); acc[3] += bf_hi(h.y) + bf_hi(l.y);
  acc[4] += bf_lo(h.z) + bf_lo(l.z); acc[5] += bf_hi(h.z) + bf_hi(l.z);
  acc[6] += bf_lo(h.w) + bf_lo(l.w); acc[7] += bf_hi(h.w) + bf_hi(l.w);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// hi = bf16(c); lo = bf16(c - hi) (c - hi is exact in FP32).
__device__ __forceinline__ void split_row(const float (&c)[8], uint4* hi, uint4* lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = pack_bf16(c[2 * q], c[2 * q + 1]);
    l[q] = pack_bf16(c[2 * q] - bf_lo(h[q]), c[2 * q + 1] - bf_hi(h[q]));
  }
  *hi = make_uint4(h[0], h[1], h[2], h[3]);
  if (lo) *lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// streaming (evict-first) store: intermBuf and carries must not push the
// segment's C rows out of L2
__device__ __forceinline__ void store_row(float* dst, const float (&a)[8]) {
  float4* p = reinterpret_cast<float4*>(dst);
  __stcs(p, make_float4(a[0], a[1], a[2], a[3]));
  __stcs(p + 1, make_float4(a[4], a[5], a[6], a[7]));
}

__device__ __forceinline__ void load_row(const float* src, float (&a)[8]) {
  const float4* p = reinterpret_cast<const float4*>(src);
  const float4 x = __ldcs(p), y = __ldcs(p + 1);
  a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
  a[4] = y.x; a[5] = y.y; a[6] = y.z; a[7] = y.w;
}

__device__ __forceinline__ uint32_t pick(const uint4& v, int c) {
  return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------------------
// Gather (Algorithm 3, 64-wide).  Octet o takes chunks o, o + #octets, ...:
// all octets sweep the chunks in segment order together, so the C rows read
// at any moment belong to one or two segments' source slices.
// ---------------------------------------------------------------------------
template <int PLANES>
__global__ void __launch_bounds__(kThreads, 6)
ppr_gather_kernel(const uint32_t* __restrict__ colf, const PprSeg* __restrict__ segs,
                  const int2* __restrict__ chunks, int64_t nchunks,
                  const uint4* __restrict__ c_hi, const uint4* __restrict__ c_lo,
                  float* __restrict__ interm, float* __restrict__ carry) {
  // edges whose rows are loaded together: one with two planes (more resident
  // warps hide the latency better than more loads per warp)
  constexpr int U = 2 / PLANES;
  const int lane8 = threadIdx.x & 7;
  const unsigned omask = 0xffu << (threadIdx.x & 24);
  const int64_t noct = ((int64_t)gridDim.x * blockDim.x) >> 3;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; c < nchunks;
       c += noct) {
    const int2 ch = __ldg(chunks + c);
    const PprSeg sg = segs[ch.y];
    const int64_t el = (c - sg.chunk0) * kChunk;
    const int n = (int)min((int64_t)kChunk, (int64_t)sg.E - el);
    const uint4* cf = reinterpret_cast<const uint4*>(colf + sg.cstart + el);
    const uint4* hb = c_hi + (int64_t)sg.lo * 8 + lane8;
    const uint4* lb = c_lo + (int64_t)sg.lo * 8 + lane8;
    int32_t row = ch.x;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    uint32_t last = kRowEnd;
    for (int sb = 0; sb < n; sb += 32) {
      const int m = min(32, n - sb);
      uint4 f4 = make_uint4(0u, 0u, 0u, 0u);
      if (4 * lane8 < m) f4 = __ldcs(cf + (sb >> 2) + lane8);
      for (int g = 0; g < m; g += 4) {  // the 4 edges held by octet lane g / 4
#pragma unroll
        for (int u0 = 0; u0 < 4; u0 += U) {
          uint32_t f[U];
          uint4 h[U], l[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            f[u] = __shfl_sync(omask, pick(f4, u0 + u), g >> 2, 8);
            if (g + u0 + u < m) {
              const int64_t s = (int64_t)(f[u] & ~kRowEnd) * 8;
              h[u] = __ldg(hb + s);
              if (PLANES == 2) l[u] = __ldg(lb + s);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (g + u0 + u < m) {
              if (PLANES == 2) add_row2(acc, h[u], l[u]); else add_row(acc, h[u]);
              last = f[u];
              if (f[u] & kRowEnd) {
                store_row(interm + (int64_t)row * kCols + lane8 * 8, acc);
                ++row;
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
              }
            }
          }
        }
      }
    }
    if (!(last & kRowEnd)) store_row(carry + c * kCols + lane8 * 8, acc);  // open row
  }
}

// Rows that span chunks.  One octet per piece (<= 32 consecutive chunks of
// one run): it sums the pieces' carries in chunk order.  A run of one piece
// adds its sum into the row directly; otherwise each piece stores its sum and
// the last piece of the run to finish (atomic count, no waiting) adds the
// pieces' sums in piece order into the row -- deterministic, and a hub row
// spanning thousands of chunks no longer holds up one octet.
__global__ void __launch_bounds__(kThreads)
ppr_fixup_kernel(const int4* __restrict__ pieces, int64_t npieces, const int4* __restrict__ runs,
                 const float* __restrict__ carry, float* __restrict__ piece_sum,
                 unsigned* __restrict__ run_done, float* __restrict__ interm) {
  const int lane8 = threadIdx.x & 7;
  const unsigned omask = 0xffu << (threadIdx.x & 24);
  const int64_t noct = ((int64_t)gridDim.x * blockDim.x) >> 3;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; p < npieces;
       p += noct) {
    const int4 pc = __ldg(pieces + p);  // (first chunk, chunks, run)
    const int4 rn = __ldg(runs + pc.z); // (row, first piece, pieces)
    float sum[8], x[8];
    load_row(carry + (int64_t)pc.x * kCols + lane8 * 8, sum);
    for (int j = 1; j < pc.y; ++j) {
      load_row(carry + ((int64_t)pc.x + j) * kCols + lane8 * 8, x);
#pragma unroll
      for (int q = 0; q < 8; ++q) sum[q] += x[q];
    }
    float* dst = interm + (int64_t)rn.x * kCols + lane8 * 8;
    if (rn.z == 1) {
      load_row(dst, x);
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] += sum[q];
      store_row(dst, x);
      continue;
    }
    store_row(piece_sum + p * kCols + lane8 * 8, sum);
    __threadfence();
    __syncwarp(omask);
    unsigned prev = 0;
    if (lane8 == 0) prev = atomicAdd(run_done + pc.z, 1u);
    prev = __shfl_sync(omask, prev, 0, 8);
    if (prev != (unsigned)rn.z - 1) continue;  // not the run's last piece
    __threadfence();
    float tot[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) tot[q] = 0.0f;
    for (int j = 0; j < rn.z; ++j) {
      const float4* ps =
          reinterpret_cast<const float4*>(piece_sum + ((int64_t)rn.y + j) * kCols + lane8 * 8);
      const float4 u = __ldcg(ps), w = __ldcg(ps + 1);
      tot[0] += u.x; tot[1] += u.y; tot[2] += u.z; tot[3] += u.w;
      tot[4] += w.x; tot[5] += w.y; tot[6] += w.z; tot[7] += w.w;
    }
    load_row(dst, x);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] += tot[q];
    store_row(dst, x);
    if (lane8 == 0) run_done[pc.z] = 0u;  // ready for the next iteration
  }
}

// ---------------------------------------------------------------------------
// Merge (Algorithm 4, destination-major) fused with the personalised update.
// ---------------------------------------------------------------------------
struct MergeArgs {
  const int32_t* dst_off;
  const int32_t* dst_rows;
  const float* interm;
  const float* inv;
  const int32_t* seeds;
  const uint32_t* seed_bits;
  uint4* c_hi;
  uint4* c_lo;
  float* r_out;        // NULL: R' not written
  const float* r_old;  // NULL: no residual
  double* D;           // [64] in: D of the previous iterate; out: D'
  double* resid;       // [64] or NULL
  double* partials;
  unsigned* counter;
  float d;
  int32_t V;
};

template <int PLANES, bool RESID>
__global__ void __launch_bounds__(kThreads, 4)
ppr_merge_kernel(MergeArgs a) {
  __shared__ float s_tele[kCols];
  __shared__ int32_t s_seed[kCols];
  __shared__ double s_red[kThreads / 32][2][kCols];
  __shared__ bool s_last;
  if (threadIdx.x < kCols) {
    s_tele[threadIdx.x] =
        (float)((1.0 - (double)a.d) + (double)a.d * a.D[threadIdx.x]);
    s_seed[threadIdx.x] = a.seeds[threadIdx.x];
  }
  __syncthreads();
  const int lane8 = threadIdx.x & 7;
  const unsigned omask = 0xffu << (threadIdx.x & 24);
  const int64_t noct = ((int64_t)gridDim.x * blockDim.x) >> 3;
  const int64_t ntask = ((int64_t)a.V + kTask - 1) / kTask;
  double dsum[8], rsum[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) dsum[q] = rsum[q] = 0.0;
  const float4* in4 = reinterpret_cast<const float4*>(a.interm);
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; t < ntask; t += noct) {
    const int64_t v0 = t * kTask;
    const int nv = (int)min((int64_t)kTask, (int64_t)a.V - v0);
    // row-list offsets and reciprocal degrees of the task's destinations
    const int32_t off_a = __ldg(a.dst_off + v0 + min(lane8, nv));
    const int32_t off_b = __ldg(a.dst_off + v0 + min(8 + lane8, nv));
    const float inv_a = lane8 < nv ? __ldg(a.inv + v0 + lane8) : 0.0f;
    const float inv_b = 8 + lane8 < nv ? __ldg(a.inv + v0 + 8 + lane8) : 0.0f;
    const uint32_t sbits = __ldg(a.seed_bits + (v0 >> 5)) >> (v0 & 31);
    const int32_t o_end = __ldg(a.dst_off + v0 + nv);
    float dpart[8], rpart[8], acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) dpart[q] = rpart[q] = acc[q] = 0.0f;
    int i = 0;  // destination being accumulated
    auto off_of = [&](int j) -> int32_t {  // start of destination j's rows, j in [0, nv]
      const int32_t x = __shfl_sync(omask, off_a, j & 7, 8);
      const int32_t y = __shfl_sync(omask, off_b, j & 7, 8);
      return j >= nv ? o_end : j < 8 ? x : y;
    };
    auto finish = [&](int j) {  // update of destination v0 + j from acc
      const int64_t v = v0 + j;
      const float iv = __shfl_sync(omask, j < 8 ? inv_a : inv_b, j & 7, 8);
      float r[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) r[q] = a.d * acc[q];
      if ((sbits >> j) & 1u) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (s_seed[lane8 * 8 + q] == (int32_t)v) r[q] += s_tele[lane8 * 8 + q];
      }
      if (iv != 0.0f) {
        float c[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = r[q] * iv;
        uint4 h, l;
        split_row(c, &h, PLANES == 2 ? &l : nullptr);
        __stcs(a.c_hi + v * 8 + lane8, h);
        if (PLANES == 2) __stcs(a.c_lo + v * 8 + lane8, l);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) dpart[q] += r[q];
      }
      if (a.r_out) {
        float4* p = reinterpret_cast<float4*>(a.r_out + v * kCols + lane8 * 8);
        __stcs(p, make_float4(r[0], r[1], r[2], r[3]));
        __stcs(p + 1, make_float4(r[4], r[5], r[6], r[7]));
      }
      if (RESID) {
        float o[8];
        load_row(a.r_old + v * kCols + lane8 * 8, o);
#pragma unroll
        for (int q = 0; q < 8; ++q) rpart[q] += fabsf(r[q] - o[q]);
      }
    };
    const int32_t o_lo = off_of(0);
    int32_t iend = off_of(1);
    constexpr int G = 2;  // intermBuf rows loaded together (4 blocks per SM fit)
    for (int32_t p = o_lo; p < o_end; p += G) {
      int32_t rr[G];
      float4 x[G], y[G];
#pragma unroll
      for (int u = 0; u < G; ++u) rr[u] = p + u < o_end ? __ldg(a.dst_rows + p + u) : 0;
#pragma unroll
      for (int u = 0; u < G; ++u) {
        if (p + u < o_end) {
          x[u] = __ldcs(in4 + (int64_t)rr[u] * (kCols / 4) + lane8 * 2);
          y[u] = __ldcs(in4 + (int64_t)rr[u] * (kCols / 4) + lane8 * 2 + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        if (p + u < o_end) {
          while (p + u >= iend) {  // rows of destination i are done
            finish(i);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
            ++i;
            iend = off_of(i + 1);
          }
          acc[0] += x[u].x; acc[1] += x[u].y; acc[2] += x[u].z; acc[3] += x[u].w;
          acc[4] += y[u].x; acc[5] += y[u].y; acc[6] += y[u].z; acc[7] += y[u].w;
        }
      }
    }
    for (; i < nv; ++i) {
      finish(i);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      dsum[q] += (double)dpart[q];
      if (RESID) rsum[q] += (double)rpart[q];
    }
  }
  // per-column partials: octets of a warp, then warps of the block
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], 8);
    dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], 16);
    if (RESID) {
      rsum[q] += __shfl_xor_sync(0xffffffffu, rsum[q], 8);
      rsum[q] += __shfl_xor_sync(0xffffffffu, rsum[q], 16);
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane < 8) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      s_red[w][0][lane * 8 + q] = dsum[q];
      s_red[w][1][lane * 8 + q] = rsum[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * kCols) {
    const int which = threadIdx.x / kCols, j = threadIdx.x % kCols;
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += s_red[q][which][j];
    a.partials[(int64_t)blockIdx.x * 2 * kCols + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 2 * kCols) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b)
      s += __ldcg(a.partials + (int64_t)b * 2 * kCols + threadIdx.x);
    if (threadIdx.x < kCols) a.D[threadIdx.x] = s;
    else if (RESID && a.resid) a.resid[threadIdx.x - kCols] = s;
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

// ---------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------
__global__ void ppr_chunks_kernel(const int32_t* __restrict__ rp, const int64_t* __restrict__ meta,
                                  const PprSeg* __restrict__ segs, int k, int64_t nchunks,
                                  int2* __restrict__ chunks) {
  // meta: row_base[k+1], edge_base[k+1] of the segmented graph
  const int64_t* row_base = meta;
  const int64_t* edge_base = meta + (k + 1);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    int s0 = 0, s1 = k;  // last segment with chunk0 <= c (and edges)
    while (s1 - s0 > 1) {
      const int mid = (s0 + s1) >> 1;
      if (segs[mid].chunk0 <= c) s0 = mid; else s1 = mid;
    }
    while (s0 + 1 < k && segs[s0 + 1].chunk0 <= c) ++s0;
    const int64_t e = edge_base[s0] + (c - segs[s0].chunk0) * kChunk;
    int64_t lo = row_base[s0], hi = row_base[s0 + 1];  // last row with rp[row] <= e
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rp[mid] <= e) lo = mid + 1; else hi = mid;
    }
    chunks[c] = make_int2((int32_t)(lo - 1), s0);
  }
}

// The row open at each chunk's end (-1 when the chunk ends a row): the
// subgraph row of the chunk's last edge, if that row continues past it.
__global__ void carry_rows_kernel(const int32_t* __restrict__ rp, const int64_t* __restrict__ meta,
                                  const PprSeg* __restrict__ segs, const int2* __restrict__ chunks,
                                  int k, int64_t nchunks, int32_t* __restrict__ carry_row) {
  const int64_t* row_base = meta;
  const int64_t* edge_base = meta + (k + 1);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int s = chunks[c].y;
    const int64_t el = (c - segs[s].chunk0) * kChunk;
    const int64_t n = min((int64_t)kChunk, (int64_t)segs[s].E - el);
    const int64_t e = edge_base[s] + el + n - 1;  // global index of the chunk's last edge
    int64_t lo = row_base[s], hi = row_base[s + 1];  // last row with rp[row] <= e
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rp[mid] <= e) lo = mid + 1; else hi = mid;
    }
    const int64_t row = lo - 1;
    carry_row[c] = (int64_t)rp[row + 1] - 1 > e ? (int32_t)row : -1;
  }
}

__global__ void count_dst_kernel(const int32_t* __restrict__ idx_map, int64_t rows,
                                 int32_t* __restrict__ cnt) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + idx_map[r], 1);
}

__global__ void narrow_kernel(const int64_t* __restrict__ in, int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

// Rows of one segment: their destinations are distinct, so each takes the
// next free slot of its destination's list without collisions; segments
// are filled in order, so every list is in segment order.
__global__ void fill_dst_kernel(const int32_t* __restrict__ idx_map, int64_t r0, int64_t r1,
                                const int32_t* __restrict__ off, int32_t* __restrict__ fill,
                                int32_t* __restrict__ dst_rows) {
  for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx_map[r];
    dst_rows[off[v] + fill[v]] = (int32_t)r;
    fill[v] += 1;
  }
}

__global__ void ppr_seed_kernel(const float* __restrict__ inv, const int32_t* __restrict__ seeds,
                                __nv_bfloat16* __restrict__ c_hi, __nv_bfloat16* __restrict__ c_lo,
                                uint32_t* __restrict__ seed_bits, double* __restrict__ D) {
  const int j = threadIdx.x;
  if (j >= kCols) return;
  const int32_t s = seeds[j];
  const float c = inv[s];  // R_0 = one-hot at the seed: C = 1 / outdeg
  const __nv_bfloat16 h = __float2bfloat16_rn(c);
  c_hi[(int64_t)s * kCols + j] = h;
  if (c_lo) c_lo[(int64_t)s * kCols + j] = __float2bfloat16_rn(c - __bfloat162float(h));
  atomicOr(seed_bits + (s >> 5), 1u << (s & 31));
  D[j] = c == 0.0f ? 1.0 : 0.0;
}

int merge_launch(cg_ppr* p, const float* inv, double damping, float* r_out, const float* r_old,
                 double* resid, cudaStream_t s) {
  MergeArgs a;
  a.dst_off = p->dst_off;
  a.dst_rows = p->dst_rows;
  a.interm = p->interm;
  a.inv = inv;
  a.seeds = p->seeds;
  a.seed_bits = p->seed_bits;
  a.c_hi = p->c_hi;
  a.c_lo = p->c_lo;
  a.r_out = r_out;
  a.r_old = r_old;
  a.D = p->D;
  a.resid = resid;
  a.partials = p->partials;
  a.counter = p->counter;
  a.d = (float)damping;
  a.V = p->V;
  const bool res = r_old != nullptr;
  if (p->planes == 2) {
    if (res) ppr_merge_kernel<2, true><<<p->merge_grid, kThreads, 0, s>>>(a);
    else ppr_merge_kernel<2, false><<<p->merge_grid, kThreads, 0, s>>>(a);
  } else {
    if (res) ppr_merge_kernel<1, true><<<p->merge_grid, kThreads, 0, s>>>(a);
    else ppr_merge_kernel<1, false><<<p->merge_grid, kThreads, 0, s>>>(a);
  }
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int gather_launch(cg_ppr* p, cudaStream_t s) {
  if (p->nchunks == 0) return CG_OK;
  const SegPlan& sp = p->seg->plan;
  if (p->planes == 2)
    ppr_gather_kernel<2><<<p->gather_grid, kThreads, 0, s>>>(
        sp.colf, p->segs, p->chunks, p->nchunks, p->c_hi, p->c_lo, p->interm, p->carry);
  else
    ppr_gather_kernel<1><<<p->gather_grid, kThreads, 0, s>>>(
        sp.colf, p->segs, p->chunks, p->nchunks, p->c_hi, p->c_hi, p->interm, p->carry);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int fixup_launch(cg_ppr* p, cudaStream_t s) {
  if (p->npieces == 0) return CG_OK;
  ppr_fixup_kernel<<<grid_for(p->npieces * 8, kThreads, 8), kThreads, 0, s>>>(
      p->pieces, p->npieces, p->runs, p->carry, p->piece_sum, p->run_done, p->interm);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

void ppr_free(cg_ppr* p) {
  ppr_dense_free(p);
  cudaFree(p->segs);
  cudaFree(p->chunks);
  cudaFree(p->carry);
  cudaFree(p->pieces);
  cudaFree(p->runs);
  cudaFree(p->piece_sum);
  cudaFree(p->run_done);
  cudaFree(p->dst_off);
  cudaFree(p->dst_rows);
  cudaFree(p->interm);
  cudaFree(p->c_hi);
  cudaFree(p->c_lo);
  cudaFree(p->r_prev);
  cudaFree(p->seeds);
  cudaFree(p->seed_bits);
  cudaFree(p->D);
  cudaFree(p->partials);
  cudaFree(p->counter);
  delete p;
}

template <class T>
cudaError_t alloc(T** ptr, int64_t n, int64_t* total) {
  const size_t b = sizeof(T) * (size_t)(n > 0 ? n : 1);
  *total += (int64_t)b;
  return cudaMalloc((void**)ptr, b);
}

int ppr_build(cg_ppr* p, cudaStream_t s) {
  const cg_segmented* g = p->seg;
  const SegPlan& sp = g->plan;
  const int k = g->k;
  int64_t& B = p->bytes;
  // segment table and gather chunks
  std::vector<PprSeg> hs(k > 0 ? k : 1);
  int64_t nch = 0;
  for (int q = 0; q < k; ++q) {
    hs[q].cstart = sp.h_cstart[q];
    hs[q].chunk0 = nch;
    hs[q].lo = (int32_t)sp.src_bounds[q];
    hs[q].E = (int32_t)(sp.edge_base[q + 1] - sp.edge_base[q]);
    nch += ceil_div(hs[q].E, kChunk);
  }
  p->nchunks = nch;
  CG_CUDA(alloc(&p->segs, k, &B));
  CG_CUDA(cudaMemcpyAsync(p->segs, hs.data(), sizeof(PprSeg) * k, cudaMemcpyHostToDevice, s));
  CG_CUDA(alloc(&p->chunks, nch, &B));
  CG_CUDA(alloc(&p->carry, nch * kCols, &B));
  if (nch > 0) {
    ppr_chunks_kernel<<<grid_for(nch, 256), 256, 0, s>>>(sp.rp32, sp.meta, p->segs, k, nch,
                                                          p->chunks);
    CG_LAUNCH_CHECK();
    // runs of carries (static) cut into pieces of <= 32 chunks
    int32_t* crow = nullptr;
    CG_CUDA(cudaMallocAsync((void**)&crow, sizeof(int32_t) * (size_t)nch, s));
    carry_rows_kernel<<<grid_for(nch, 256), 256, 0, s>>>(sp.rp32, sp.meta, p->segs, p->chunks,
                                                         k, nch, crow);
    cudaError_t ce = cudaGetLastError();
    std::vector<int32_t> hc((size_t)nch);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(hc.data(), crow, sizeof(int32_t) * (size_t)nch,
                           cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFreeAsync(crow, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppr_batched_create", __FILE__, __LINE__);
    std::vector<int4> hp, hr;
    for (int64_t c = 0; c < nch;) {
      if (hc[c] < 0) { ++c; continue; }
      int64_t e = c + 1;
      while (e < nch && hc[e] == hc[c]) ++e;
      const int32_t run = (int32_t)hr.size(), p0 = (int32_t)hp.size();
      for (int64_t x = c; x < e; x += 32)
        hp.push_back(make_int4((int32_t)x, (int32_t)std::min<int64_t>(32, e - x), run, 0));
      hr.push_back(make_int4(hc[c], p0, (int32_t)hp.size() - p0, 0));
      c = e;
    }
    p->npieces = (int64_t)hp.size();
    p->nruns = (int64_t)hr.size();
    CG_CUDA(alloc(&p->pieces, p->npieces, &B));
    CG_CUDA(alloc(&p->runs, p->nruns, &B));
    CG_CUDA(alloc(&p->piece_sum, p->npieces * kCols, &B));
    CG_CUDA(alloc(&p->run_done, p->nruns, &B));
    if (p->npieces > 0) {
      CG_CUDA(cudaMemcpyAsync(p->pieces, hp.data(), sizeof(int4) * hp.size(),
                              cudaMemcpyHostToDevice, s));
      CG_CUDA(cudaMemcpyAsync(p->runs, hr.data(), sizeof(int4) * hr.size(),
                              cudaMemcpyHostToDevice, s));
      CG_CUDA(cudaMemsetAsync(p->run_done, 0, sizeof(unsigned) * hr.size(), s));
      CG_CUDA(cudaStreamSynchronize(s));  // hp / hr go out of scope
    }
  }
  // destination-major row lists
  const int32_t V = p->V;
  int32_t* cnt = nullptr;
  int64_t* off64 = nullptr;
  CG_CUDA(alloc(&p->dst_off, (int64_t)V + 1, &B));
  CG_CUDA(alloc(&p->dst_rows, p->rows, &B));
  CG_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int32_t) * (size_t)V, s));
  cudaError_t e = cudaMallocAsync((void**)&off64, sizeof(int64_t) * ((size_t)V + 1), s);
  int st = CG_OK;
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)V, s);
  if (e == cudaSuccess && p->rows > 0) {
    count_dst_kernel<<<grid_for(p->rows, 256), 256, 0, s>>>(g->idx_map, p->rows, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) st = exclusive_scan_i32_to_i64(cnt, off64, V, s);
  if (e == cudaSuccess && st == CG_OK) {
    narrow_kernel<<<grid_for((int64_t)V + 1, 256), 256, 0, s>>>(off64, (int64_t)V + 1, p->dst_off);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && st == CG_OK) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)V, s);
  for (int q = 0; q < k && e == cudaSuccess && st == CG_OK; ++q) {
    const int64_t r0 = g->row_base[q], r1 = g->row_base[q + 1];
    if (r1 > r0) {
      fill_dst_kernel<<<grid_for(r1 - r0, 256), 256, 0, s>>>(g->idx_map, r0, r1, p->dst_off, cnt,
                                                              p->dst_rows);
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(off64, s);
  if (st != CG_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "ppr_batched_create", __FILE__, __LINE__);
  // iteration state
  CG_CUDA(alloc(&p->interm, p->rows * kCols, &B));
  CG_CUDA(alloc(&p->c_hi, (int64_t)V * 8, &B));
  if (p->planes == 2) CG_CUDA(alloc(&p->c_lo, (int64_t)V * 8, &B));
  CG_CUDA(alloc(&p->r_prev, (int64_t)V * kCols, &B));
  CG_CUDA(alloc(&p->seeds, kCols, &B));
  CG_CUDA(alloc(&p->seed_bits, ceil_div(V, 32), &B));
  CG_CUDA(alloc(&p->D, kCols, &B));
  // launch shapes: whole waves of resident blocks
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  int per_sm = 0;
  CG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, p->planes == 2 ? ppr_merge_kernel<2, true> : ppr_merge_kernel<1, true>, kThreads,
      0));
  p->merge_grid = di.sm_count * (per_sm > 0 ? per_sm : 1);
  CG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, p->planes == 2 ? ppr_gather_kernel<2> : ppr_gather_kernel<1>, kThreads, 0));
  p->gather_grid = di.sm_count * (per_sm > 0 ? per_sm : 1);
  CG_CUDA(alloc(&p->partials, (int64_t)p->merge_grid * 2 * kCols, &B));
  CG_CUDA(alloc(&p->counter, 1, &B));
  CG_CUDA(cudaMemsetAsync(p->counter, 0, sizeof(unsigned), s));
  CG_CUDA(cudaStreamSynchronize(s));
  return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int ppr_batched_create(const cg_segmented* seg, int32_t planes, cg_ppr** out,
                       cudaStream_t stream) {
  CG_ARG(out != nullptr, "ppr_batched_create: out is NULL");
  *out = nullptr;
  CG_ARG(seg != nullptr, "ppr_batched_create: null segmented graph");
  CG_ARG(planes == 1 || planes == 2, "ppr_batched_create: planes must be 1 or 2 (got %d)",
         planes);
  int dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  CG_ARG(dev == seg->device, "ppr_batched_create: the segmented graph lives on device %d, "
         "current device is %d", seg->device, dev);
  cg_ppr* p = new cg_ppr();
  p->device = dev;
  p->seg = seg;
  p->V = seg->V;
  p->k = seg->k;
  p->rows = seg->rows;
  p->planes = planes;
  const int st = ppr_build(p, stream);
  if (st != CG_OK) {
    cudaStreamSynchronize(stream);
    ppr_free(p);
    return st;
  }
  *out = p;
  return CG_OK;
}

int ppr_batched_destroy(cg_ppr* p) {
  if (!p) return CG_OK;
  cudaDeviceSynchronize();
  ppr_free(p);
  return CG_OK;
}

int ppr_batched_bytes(const cg_ppr* p, int64_t* bytes, int64_t* chunks) {
  CG_ARG(p != nullptr, "ppr_batched_bytes: null handle");
  if (bytes) *bytes = p->bytes;
  if (chunks) *chunks = p->nchunks;
  return CG_OK;
}

int ppr_batched_init(cg_ppr* p, const float* inv, const int32_t* host_seeds,
                     cudaStream_t stream) {
  CG_ARG(p && inv && host_seeds, "ppr_batched_init: null argument");
  for (int j = 0; j < kCols; ++j)
    CG_ARG(host_seeds[j] >= 0 && host_seeds[j] < p->V,
           "ppr_batched_init: seed %d of column %d outside [0, %d)", host_seeds[j], j, p->V);
  const size_t plane = sizeof(uint4) * 8 * (size_t)p->V;
  CG_CUDA(cudaMemcpyAsync(p->seeds, host_seeds, sizeof(int32_t) * kCols, cudaMemcpyHostToDevice,
                          stream));
  CG_CUDA(cudaMemsetAsync(p->c_hi, 0, plane, stream));
  if (p->c_lo) CG_CUDA(cudaMemsetAsync(p->c_lo, 0, plane, stream));
  CG_CUDA(cudaMemsetAsync(p->seed_bits, 0, sizeof(uint32_t) * (size_t)ceil_div(p->V, 32),
                          stream));
  ppr_seed_kernel<<<1, kCols, 0, stream>>>(inv, p->seeds, reinterpret_cast<__nv_bfloat16*>(p->c_hi),
                                           reinterpret_cast<__nv_bfloat16*>(p->c_lo),
                                           p->seed_bits, p->D);
  CG_LAUNCH_CHECK();
  CG_TRY(ppr_dense_pack(p, stream));
  // host_seeds may go out of scope on return
  CG_CUDA(cudaStreamSynchronize(stream));
  p->seeded = true;
  return CG_OK;
}

int ppr_batched_step(cg_ppr* p, const float* inv, double damping, int32_t phases,
                     const float* rank_old, float* rank_out, double* resid,
                     cudaStream_t stream) {
  CG_ARG(p && inv, "ppr_batched_step: null argument");
  CG_ARG(p->seeded, "ppr_batched_step: call ppr_batched_init first");
  CG_ARG(damping >= 0.0 && damping <= 1.0, "ppr_batched_step: damping must be in [0, 1]");
  CG_ARG(phases >= 0 && phases <= 15, "ppr_batched_step: phases must be in [0, 15]");
  CG_ARG(!resid || rank_old, "ppr_batched_step: the residual needs rank_old");
  CG_ARG(!rank_old || rank_out, "ppr_batched_step: rank_old needs rank_out");
  CG_ARG(!rank_out || (const float*)rank_out != rank_old,
         "ppr_batched_step: rank_out must not alias rank_old");
  if (phases & 1) CG_TRY(gather_launch(p, stream));
  if (phases & 8) CG_TRY(ppr_dense_launch(p, stream));  // the hub block's rows (if attached)
  if (phases & 2) CG_TRY(fixup_launch(p, stream));
  if (phases & 4) {
    CG_TRY(merge_launch(p, inv, damping, rank_out, rank_old, resid, stream));
    CG_TRY(ppr_dense_pack(p, stream));
  }
  return CG_OK;
}

int ppr_batched_iterate(cg_ppr* p, const float* inv, double damping, int32_t iterations,
                        float* rank_out, double* resid, cudaStream_t stream) {
  CG_ARG(p && inv, "ppr_batched_iterate: null argument");
  CG_ARG(iterations >= 1, "ppr_batched_iterate: iterations must be >= 1");
  CG_ARG(!resid || (iterations >= 2 && rank_out),
         "ppr_batched_iterate: the residual needs iterations >= 2 and rank_out");
  for (int t = 0; t < iterations; ++t) {
    const bool last = t == iterations - 1;
    const bool before_last = t == iterations - 2 && resid;
    float* r_out = last ? rank_out : before_last ? p->r_prev : nullptr;
    const float* r_old = last && resid ? p->r_prev : nullptr;
    CG_TRY(ppr_batched_step(p, inv, damping, 15, r_old, r_out, last ? resid : nullptr, stream));
  }
  return CG_OK;
}

}  // extern "C"
