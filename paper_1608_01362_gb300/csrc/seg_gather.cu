// Flagged-edge segment gather: plan construction and the kernel.
#include <algorithm>

#include "seg_gather.cuh"

namespace cg {
namespace {

__device__ __forceinline__ int last_le(const int64_t* a, int n, int64_t v) {
  // last index q in [0, n) with a[q] <= v (a ascending, a[0] <= v)
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// One warp per subgraph row: copy its sources, as indices local to their
// segment, into the padded layout and flag the last one.
__global__ void colf_fill_kernel(const int32_t* __restrict__ col, const int64_t* __restrict__ rp,
                                 int64_t rows, const int64_t* __restrict__ row_base,
                                 const int64_t* __restrict__ edge_base,
                                 const int64_t* __restrict__ cstart,
                                 const int64_t* __restrict__ bounds, int k,
                                 uint32_t* __restrict__ colf) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += nw) {
    const int s = last_le(row_base, k + 1, i);
    const int64_t lo = rp[i], hi = rp[i + 1];
    const int64_t shift = cstart[s] - edge_base[s];
    const int32_t src0 = (int32_t)bounds[s];
    for (int64_t e = lo + lane; e < hi; e += 32)
      colf[e + shift] = (uint32_t)(col[e] - src0) | (e == hi - 1 ? kRowEndFlag : 0u);
  }
}

__global__ void export_col_kernel(const uint32_t* __restrict__ colf,
                                  const int32_t* __restrict__ rp, int64_t rows,
                                  const int64_t* __restrict__ row_base,
                                  const int64_t* __restrict__ edge_base,
                                  const int64_t* __restrict__ cstart,
                                  const int64_t* __restrict__ bounds, int k,
                                  int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += nw) {
    const int s = last_le(row_base, k + 1, i);
    const int64_t shift = cstart[s] - edge_base[s];
    const int32_t src0 = (int32_t)bounds[s];
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32)
      col[e] = src0 + (int32_t)(colf[e + shift] & ~kRowEndFlag);
  }
}

// The row open at each chunk's end (-1 when the chunk ends a row): the
// subgraph row of the chunk's last edge, if that row continues past it.
__global__ void open_row_kernel(const int32_t* __restrict__ rp,
                                const int64_t* __restrict__ row_base,
                                const int64_t* __restrict__ edge_base,
                                const int64_t* __restrict__ chunk_base, int k, int m, int chunk_a,
                                int chunk_b, int64_t nchunks, int32_t* __restrict__ open_row) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int s = last_le(chunk_base, k + 1, c);
    const int64_t size = s < m ? chunk_a : chunk_b;
    const int64_t e0 = edge_base[s] + (c - chunk_base[s]) * size;
    const int64_t e = min(e0 + size, edge_base[s + 1]) - 1;  // the chunk's last edge
    int64_t lo = row_base[s], hi = row_base[s + 1];  // last row with rp[row] <= e
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rp[mid] <= e) lo = mid + 1; else hi = mid;
    }
    open_row[c] = (int64_t)rp[lo] - 1 > e ? (int32_t)(lo - 1) : -1;
  }
}

// Completion of the rows that span chunks, one thread per piece (<= 32
// consecutive chunks of one run of carries on the same row).  A one-piece
// run folds its carries into the row directly; otherwise every piece stores
// its fold and the last piece of the run to finish (an atomic count, no
// waiting) folds the pieces in order into the row.  Deterministic, and a hub
// row spanning many chunks is spread over many threads.
template <class Op>
__global__ void seg_fixup_kernel(const int4* __restrict__ pieces, int64_t npieces,
                                 const int4* __restrict__ runs,
                                 const typename Op::T* __restrict__ carry,
                                 typename Op::T* __restrict__ psum, unsigned* __restrict__ done,
                                 typename Op::T* __restrict__ out) {
  using T = typename Op::T;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npieces;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int4 pc = pieces[p];  // (first chunk, chunks, run)
    const int4 rn = runs[pc.z]; // (row, first piece, pieces)
    T v = carry[pc.x];
    for (int j = 1; j < pc.y; ++j) v = Op::op(v, carry[pc.x + j]);
    if (rn.z == 1) {
      out[rn.x] = Op::op(v, out[rn.x]);
      continue;
    }
    psum[p] = v;
    __threadfence();
    if (atomicAdd(done + pc.z, 1u) != (unsigned)rn.z - 1) continue;
    __threadfence();
    T t = __ldcg(psum + rn.y);
    for (int j = 1; j < rn.z; ++j) t = Op::op(t, __ldcg(psum + rn.y + j));
    out[rn.x] = Op::op(t, out[rn.x]);
    done[pc.z] = 0u;  // ready for the next pass
  }
}

// Subgraph row of each chunk's first edge (segments [0, m) use chunks of
// chunk_a edges, the others chunks of chunk_b).
__global__ void first_row_kernel(const int32_t* __restrict__ rp,
                                 const int64_t* __restrict__ row_base,
                                 const int64_t* __restrict__ edge_base,
                                 const int64_t* __restrict__ chunk_base, int k, int m, int chunk_a,
                                 int chunk_b, int64_t nchunks, int32_t* __restrict__ first_row) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int s = last_le(chunk_base, k + 1, c);
    const int64_t e = edge_base[s] + (c - chunk_base[s]) * (s < m ? chunk_a : chunk_b);
    int64_t lo = row_base[s], hi = row_base[s + 1];  // last row with rp[row] <= e
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rp[mid] <= e) lo = mid + 1; else hi = mid;
    }
    first_row[c] = (int32_t)(lo - 1);
  }
}

// One L1/L2 chunk: 256 edges of segment-local chunk j (global chunk c) of a
// segment whose sources start at lo; lane l holds edges [8l, 8l + 8).
constexpr int kCachedIPL = 8;
constexpr int kCachedChunk = 32 * kCachedIPL;  // 256 edges

template <class Op>
__device__ __forceinline__ void cached_chunk(const uint32_t* __restrict__ colf,
                                             const typename Op::T* __restrict__ x, int32_t nx,
                                             int32_t lo, int32_t Es, int32_t cstart, int32_t j,
                                             int32_t c, int32_t frow,
                                             typename Op::T* __restrict__ out,
                                             typename Op::T* __restrict__ carry) {
  using T = typename Op::T;
  constexpr int IPL = kCachedIPL;
  constexpr int CHUNK = kCachedChunk;
  const int lane = threadIdx.x & 31;
  const int32_t e0 = j * CHUNK;
  const int n = Es - e0 < CHUNK ? Es - e0 : CHUNK;

  // 1. this lane's 8 edges (two 16-byte streaming loads; colf is padded)
  const uint4* p = reinterpret_cast<const uint4*>(colf + cstart + e0 + lane * IPL);
  const uint4 qa = __ldcs(p), qb = __ldcs(p + 1);
  const uint32_t cf[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
  T v[IPL];
  uint32_t fl = 0;
  const int nl = n - lane * IPL;  // valid edges of this lane
#pragma unroll
  for (int u = 0; u < IPL; ++u) {
    const bool ok = u < nl;
    const int32_t src = lo + (int32_t)(cf[u] & ~kRowEndFlag);
    if (ok) fl |= (cf[u] >> 31) << u;
    v[u] = (ok && (uint32_t)src < (uint32_t)nx) ? __ldg(x + src) : Op::identity();
  }

  // 2. rows ended before this lane (exclusive warp prefix of flag counts)
  const int F = __popc(fl);
  int incl = F;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int32_t row0 = frow + (incl - F);

  // 3. sequential fold; rows that start and end in this lane are final
  T acc = Op::identity(), first_val = Op::identity();
  int nf = 0;
#pragma unroll
  for (int u = 0; u < IPL; ++u) {
    acc = Op::op(acc, v[u]);
    if (fl & (1u << u)) {
      if (nf == 0)
        first_val = acc;
      else
        out[row0 + nf] = acc;
      ++nf;
      acc = Op::identity();
    }
  }

  // 4. segmented scan of the open-row parts; completes each lane's first row
  T S = acc;
  int h = F > 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, S, o);
    const int g = __shfl_up_sync(0xffffffffu, h, o);
    if (lane >= o) {
      if (!h) S = Op::op(y, S);
      h |= g;
    }
  }
  const T P = __shfl_up_sync(0xffffffffu, S, 1);
  if (F > 0) out[row0] = lane > 0 ? Op::op(P, first_val) : first_val;

  // 5. the row open at the chunk's end (completed by the carry pieces)
  const uint32_t lf = __shfl_sync(0xffffffffu, fl, (n - 1) / IPL);
  if (lane == 31 && !((lf >> ((n - 1) % IPL)) & 1u)) carry[c] = S;
}

// The L1/L2 launch: every read of a segment in [ct_begin, ct_end) goes
// through L1/L2.  Blocks take block-groups round-robin (the grid sweeps the
// groups in order, which balances blocks when the cost per group varies).
template <class Op, int THREADS>
__global__ void __launch_bounds__(THREADS, 2048 / THREADS)
seg_gather_kernel(const uint32_t* __restrict__ colf, const typename Op::T* __restrict__ x,
                  int32_t nx, const int32_t* __restrict__ first_row,
                  const int64_t* __restrict__ seg_cstart, const int32_t* __restrict__ seg_E,
                  const int64_t* __restrict__ seg_chunk, const int32_t* __restrict__ seg_ctile,
                  const int32_t* __restrict__ seg_lo, int k, int32_t ct_begin, int32_t ct_end,
                  typename Op::T* __restrict__ out, typename Op::T* __restrict__ carry) {
  constexpr int WARPS = THREADS / 32;
  const int w = threadIdx.x >> 5;
  const int32_t my_lo = ct_begin + (int32_t)blockIdx.x;
  const int32_t step = (int32_t)gridDim.x;
  if (my_lo >= ct_end) return;
  int s;  // segment of the first group; later ones are found by stepping forward
  {
    int a = 0, b = k + 1;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (seg_ctile[mid] <= my_lo) a = mid + 1; else b = mid;
    }
    s = a - 1;
  }
  int32_t lo = 0, Es = 0, cstart = 0, cbase = 0, ctbase = 0, ctnext = -1;

  for (int32_t ct = my_lo; ct < ct_end; ct += step) {
    if (ct >= ctnext) {
      while (ct >= seg_ctile[s + 1]) ++s;
      lo = seg_lo[s];
      Es = seg_E[s];
      cstart = (int32_t)seg_cstart[s];
      cbase = (int32_t)seg_chunk[s];
      ctbase = seg_ctile[s];
      ctnext = seg_ctile[s + 1];
    }
    const int32_t j = (ct - ctbase) * WARPS + w;  // chunk of this warp within the segment
    if (j * kCachedChunk >= Es) continue;         // warp-uniform
    cached_chunk<Op>(colf, x, nx, lo, Es, cstart, j, cbase + j, first_row[cbase + j], out,
                     carry);
  }
}

// Copy n values into shared memory with many independent loads in flight per
// thread (16-byte loads when the source is 16-byte aligned), so staging a
// table costs a few memory round trips rather than one per element.
// nt: threads taking part (tid in [0, nt)).
template <typename T>
__device__ __forceinline__ void stage_table(const T* __restrict__ src, int n, T* dst, int tid,
                                            int nt) {
  static_assert(sizeof(T) == 4, "4-byte values");
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int n4 = n >> 2;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (int b = 0; b < n4; b += nt * 4) {
      uint4 r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = b + u * nt + tid;
        if (i < n4) r[u] = __ldg(s4 + i);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = b + u * nt + tid;
        if (i < n4) d4[i] = r[u];
      }
    }
    for (int i = (n4 << 2) + tid; i < n; i += nt) dst[i] = src[i];
  } else {
    for (int b = 0; b < n; b += nt * 8) {
      T r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = b + u * nt + tid;
        if (i < n) r[u] = __ldg(src + i);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = b + u * nt + tid;
        if (i < n) dst[i] = r[u];
      }
    }
  }
}

// Staged chunk stream, per 512-edge chunk (1168 bytes):
//   [0, 1024)     512 uint16 segment-local source indices, lane l's 16 edges
//                 at bytes [32l, 32l + 32)
//   [1024, 1152)  32 uint32, lane l's: bits 0-15 its row-end mask (bit u:
//                 edge u ends a row), bits 16-31 the row ends in lanes before l
//   [1152, 1156)  int32 subgraph row of the chunk's first edge
constexpr int kStagedIPL = 16;
constexpr int kStagedChunk = 32 * kStagedIPL;  // 512 edges
constexpr int kStagedChunkBytes = 2 * kStagedChunk + 64 + 64 + 16;  // 1168

// One warp per staged chunk: pack its 512 edges, the lanes' row-end masks and
// their exclusive prefix, and the chunk's first subgraph row.
__global__ void staged_fill_kernel(const uint32_t* __restrict__ colf,
                                   const int64_t* __restrict__ seg_chunk,
                                   const int64_t* __restrict__ seg_cstart,
                                   const int32_t* __restrict__ seg_E,
                                   const int32_t* __restrict__ first_row, int m,
                                   int64_t nchunks_a, uint8_t* __restrict__ cs) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks_a;
       c += nw) {
    const int s = last_le(seg_chunk, m + 1, c);
    const int64_t e_begin = (c - seg_chunk[s]) * kStagedChunk + lane * kStagedIPL;
    uint32_t packed[kStagedIPL / 2];
    uint32_t fl = 0;
#pragma unroll
    for (int u = 0; u < kStagedIPL; ++u) {
      const int64_t e = e_begin + u;
      uint32_t idx = 0;
      if (e < seg_E[s]) {
        const uint32_t wv = colf[seg_cstart[s] + e];
        idx = wv & 0xFFFFu;  // segment-local index (< 65536 for staged segments)
        fl |= (wv >> 31) << u;
      }
      if (u & 1) packed[u >> 1] |= idx << 16; else packed[u >> 1] = idx;
    }
    const int F = __popc(fl);
    int incl = F;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint8_t* base = cs + c * kStagedChunkBytes;
    uint4* dst = reinterpret_cast<uint4*>(base + lane * 32);
    dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    reinterpret_cast<uint32_t*>(base + 2 * kStagedChunk)[lane] =
        (fl & 0xFFFFu) | ((uint32_t)(incl - F) << 16);
    if (lane == 0) {
      int32_t* tail = reinterpret_cast<int32_t*>(base + 2 * kStagedChunk + 128);
      tail[0] = first_row[c];
      tail[1] = tail[2] = tail[3] = 0;
    }
  }
}

// One staged chunk whose stream words are loaded: pk (16 indices), fl (row
// ends), pre (row ends before this lane), frow (first subgraph row).
template <class Op>
__device__ __forceinline__ void staged_chunk(const uint32_t (&pk)[8], uint32_t fl, int pre,
                                             int n, int32_t c, int32_t frow,
                                             const typename Op::T* tab, uint32_t tmax,
                                             typename Op::T* __restrict__ out,
                                             typename Op::T* __restrict__ carry) {
  using T = typename Op::T;
  constexpr int IPL = kStagedIPL;
  constexpr int CHUNK = kStagedChunk;
  const int lane = threadIdx.x & 31;
  T v[IPL];
  const uint32_t tmax2 = tmax | (tmax << 16);  // both 16-bit halves clamped at once
  if (n == CHUNK) {
#pragma unroll
    for (int u = 0; u < IPL; u += 2) {
      const uint32_t q = __vminu2(pk[u >> 1], tmax2);
      v[u] = tab[q & 0xFFFFu];
      v[u + 1] = tab[q >> 16];
    }
  } else {  // a segment's last chunk: lanes past its end hold nothing
    const int nl = n - lane * IPL;
#pragma unroll
    for (int u = 0; u < IPL; u += 2) {
      const uint32_t q = __vminu2(pk[u >> 1], tmax2);
      v[u] = u < nl ? tab[q & 0xFFFFu] : Op::identity();
      v[u + 1] = u + 1 < nl ? tab[q >> 16] : Op::identity();
    }
    fl &= nl >= IPL ? 0xFFFFu : (nl <= 0 ? 0u : ((1u << nl) - 1u));
  }
  const int F = __popc(fl);
  const int32_t row0 = frow + pre;
  // sequential fold; rows that start and end in this lane are final
  T acc = Op::identity(), first_val = Op::identity();
  int nf = 0;
#pragma unroll
  for (int u = 0; u < IPL; ++u) {
    acc = Op::op(acc, v[u]);
    if (fl & (1u << u)) {
      if (nf == 0)
        first_val = acc;
      else
        out[row0 + nf] = acc;
      ++nf;
      acc = Op::identity();
    }
  }
  // the part of each lane's first row held by earlier lanes: one exchange
  // when every lane ends a row, a segmented scan otherwise
  T S = acc;
  if (!__all_sync(0xffffffffu, F > 0)) {
    int h = F > 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, S, o);
      const int g = __shfl_up_sync(0xffffffffu, h, o);
      if (lane >= o) {
        if (!h) S = Op::op(y, S);
        h |= g;
      }
    }
  }
  const T P = __shfl_up_sync(0xffffffffu, S, 1);
  if (F > 0) out[row0] = lane > 0 ? Op::op(P, first_val) : first_val;
  // the row open at the chunk's end (completed by the carry pieces)
  const uint32_t lf = __shfl_sync(0xffffffffu, fl, (n - 1) / IPL);
  if (lane == 31 && !((lf >> ((n - 1) % IPL)) & 1u)) carry[c] = S;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA; p and bytes 16-byte aligned).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void staged_load(const uint8_t* __restrict__ cs, int32_t c,
                                            uint32_t (&pk)[8], uint32_t& fl, int& pre,
                                            int32_t& frow) {
  const int lane = threadIdx.x & 31;
  const uint8_t* base = cs + (int64_t)c * kStagedChunkBytes;
  const uint4 qa = __ldcs(reinterpret_cast<const uint4*>(base + lane * 32));
  const uint4 qb = __ldcs(reinterpret_cast<const uint4*>(base + lane * 32 + 16));
  const uint32_t w = __ldcs(reinterpret_cast<const unsigned*>(base + 2 * kStagedChunk) + lane);
  fl = w & 0xFFFFu;
  pre = (int)(w >> 16);
  frow = __ldcs(reinterpret_cast<const int32_t*>(base + 2 * kStagedChunk + 128));
  pk[0] = qa.x; pk[1] = qa.y; pk[2] = qa.z; pk[3] = qa.w;
  pk[4] = qb.x; pk[5] = qb.y; pk[6] = qb.z; pk[7] = qb.w;
}

// Barrier among threads [0, nt) of the block: the whole block, or named
// barrier 1 when only the staged warps of an overlapped launch take part.
__device__ __forceinline__ void group_sync(int nt) {
  if (nt == (int)blockDim.x)
    __syncthreads();
  else
    asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
}

// The staged schedule, run by threads [0, nt) of a block: segments [0, m)
// are read from a shared-memory copy of their source values.  Work pieces
// of consecutive block-groups (nt/32 chunks each; at most `piece`, shrinking
// towards the end) are handed out in increasing order by an atomic counter
// of block-groups: a block's groups only move forward (so it stages each
// segment's table at most once) and a slow block simply takes fewer pieces.
// A warp's chunk is 512 edges of the compressed stream (lane l holds 16);
// while it works on one chunk the TMA unit prefetches its next one into L2.
template <class Op>
__device__ __forceinline__ void staged_pieces(
    const uint8_t* __restrict__ cs, const typename Op::T* __restrict__ x,
    const int32_t* __restrict__ seg_E, const int64_t* __restrict__ seg_chunk,
    const int32_t* __restrict__ seg_ctile, const int32_t* __restrict__ seg_lo,
    const int32_t* __restrict__ seg_tab, int32_t ct_end, int32_t piece,
    unsigned* __restrict__ next_piece, typename Op::T* __restrict__ out,
    typename Op::T* __restrict__ carry, typename Op::T* tab, int nt, int32_t* s_piece,
    int32_t* s_size) {
  using T = typename Op::T;
  constexpr int CHUNK = kStagedChunk;
  const int warps = nt >> 5;
  const int tid = threadIdx.x, w = tid >> 5;
  int s = 0;
  int32_t Es = 0, cbase = 0, ctbase = 0, ctnext = -1;
  uint32_t tmax = 0;

  for (;;) {
    group_sync(nt);  // everyone is done with the previous piece's s_piece
    if (tid == 0) {
      // guided self-scheduling: a piece is the remaining block-groups over
      // twice the grid, at most `piece` and at least one, so the last
      // pieces are small and the blocks finish together
      const int32_t cur = (int32_t)*(volatile unsigned*)next_piece;
      int32_t sz = (ct_end - cur) / (2 * (int32_t)gridDim.x);
      sz = sz < 1 ? 1 : (sz > piece ? piece : sz);
      *s_piece = (int32_t)atomicAdd(next_piece, (unsigned)sz);
      *s_size = sz;
    }
    group_sync(nt);
    const int32_t my_lo = *s_piece;
    if (my_lo >= ct_end) break;
    const int32_t my_hi = my_lo + *s_size < ct_end ? my_lo + *s_size : ct_end;
    for (int32_t ct = my_lo; ct < my_hi;) {
      if (ct >= ctnext) {  // a new segment (uniform across the group)
        while (ct >= seg_ctile[s + 1]) ++s;
        Es = seg_E[s];
        cbase = (int32_t)seg_chunk[s];
        ctbase = seg_ctile[s];
        ctnext = seg_ctile[s + 1];
        const int32_t lo = seg_lo[s], tn = seg_tab[s];
        tmax = tn > 0 ? (uint32_t)(tn - 1) : 0u;
        group_sync(nt);  // every warp is done reading the previous table
        stage_table<T>(x + lo, tn, tab, tid, nt);
        group_sync(nt);
      }
      const int32_t j = (ct - ctbase) * warps + w;
      if (j * CHUNK < Es) {  // warp-uniform
        const int32_t c = cbase + j;
        // ask the TMA unit to pull this warp's next chunk into L2 meanwhile
        if ((threadIdx.x & 31) == 0 && ct + 1 < my_hi && (j + warps) * CHUNK < Es)
          prefetch_l2(cs + (int64_t)(c + warps) * kStagedChunkBytes, kStagedChunkBytes);
        uint32_t pk[8], fl;
        int pre;
        int32_t frow;
        staged_load(cs, c, pk, fl, pre, frow);
        staged_chunk<Op>(pk, fl, pre, Es - j * CHUNK < CHUNK ? Es - j * CHUNK : CHUNK, c, frow,
                         tab, tmax, out, carry);
      }
      ++ct;
    }
  }
}

// The staged launch: every thread of the block runs the staged schedule.
template <class Op, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
staged_gather_kernel(const uint8_t* __restrict__ cs, const typename Op::T* __restrict__ x,
                     const int32_t* __restrict__ seg_E, const int64_t* __restrict__ seg_chunk,
                     const int32_t* __restrict__ seg_ctile, const int32_t* __restrict__ seg_lo,
                     const int32_t* __restrict__ seg_tab, int32_t ct_end, int32_t piece,
                     unsigned* __restrict__ next_piece, typename Op::T* __restrict__ out,
                     typename Op::T* __restrict__ carry) {
  using T = typename Op::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int32_t s_piece, s_size;
  staged_pieces<Op>(cs, x, seg_E, seg_chunk, seg_ctile, seg_lo, seg_tab, ct_end, piece,
                    next_piece, out, carry, reinterpret_cast<T*>(smem_raw), THREADS, &s_piece,
                    &s_size);
}

// The segment-affine staged launch (the nested form of two-level segmenting:
// the cold part of the source range, which an L2-sized segment would serve
// with random L2 reads, cut into shared-memory-sized segments).  Each block
// takes whole segments of [m, m2) from a counter, in order (heaviest first
// after clustering), stages the segment's table once and streams all its
// chunks with every warp; low-degree segments thus pay one table copy each
// instead of one per block.
template <class Op>
__global__ void __launch_bounds__(1024, 1)
affine_gather_kernel(const uint8_t* __restrict__ cs, const typename Op::T* __restrict__ x,
                     const int32_t* __restrict__ seg_E, const int64_t* __restrict__ seg_chunk,
                     const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_tab,
                     int m, int m2, unsigned* __restrict__ next_seg,
                     typename Op::T* __restrict__ out, typename Op::T* __restrict__ carry) {
  using T = typename Op::T;
  constexpr int CHUNK = kStagedChunk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);
  __shared__ int32_t s_seg;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (;;) {
    __syncthreads();  // every warp is done with the previous table and s_seg
    if (tid == 0) s_seg = m + (int32_t)atomicAdd(next_seg, 1u);
    __syncthreads();
    const int s = s_seg;
    if (s >= m2) break;
    const int32_t Es = seg_E[s], cbase = (int32_t)seg_chunk[s], tn = seg_tab[s];
    const int32_t nch = (Es + CHUNK - 1) / CHUNK;
    if (nch == 0) continue;
    stage_table<T>(x + seg_lo[s], tn, tab, tid, 1024);
    __syncthreads();
    const uint32_t tmax = tn > 0 ? (uint32_t)(tn - 1) : 0u;
    for (int32_t j = w; j < nch; j += 32) {
      const int32_t c = cbase + j;
      if (lane == 0 && j + 32 < nch)
        prefetch_l2(cs + (int64_t)(c + 32) * kStagedChunkBytes, kStagedChunkBytes);
      uint32_t pk[8], fl;
      int pre;
      int32_t frow;
      staged_load(cs, c, pk, fl, pre, frow);
      staged_chunk<Op>(pk, fl, pre, Es - j * CHUNK < CHUNK ? Es - j * CHUNK : CHUNK, c, frow, tab,
                       tmax, out, carry);
    }
  }
}

// L1/L2 chunks of segments [m, k) taken from a queue (a global counter of
// chunks, kCachedGrab at a time): a warp's successive grabs only move forward,
// so its segment is found by stepping.  The grab's chunks are prefetched into
// L2 (TMA) when it is taken.
constexpr int kCachedGrab = 4;

template <class Op>
__device__ __forceinline__ void cached_queue(
    const uint32_t* __restrict__ colf, const typename Op::T* __restrict__ x, int32_t nx,
    const int32_t* __restrict__ first_row, const int64_t* __restrict__ seg_cstart,
    const int32_t* __restrict__ seg_E, const int64_t* __restrict__ seg_chunk,
    const int32_t* __restrict__ seg_lo, int m, int k, unsigned* __restrict__ next_chunk,
    typename Op::T* __restrict__ out, typename Op::T* __restrict__ carry) {
  const int lane = threadIdx.x & 31;
  const int32_t c_begin = (int32_t)seg_chunk[m], c_end = (int32_t)seg_chunk[k];
  int s = m;
  int32_t lo = 0, Es = 0, cstart = 0, cbase = 0, cnext = -1;
  for (;;) {
    int32_t c0 = 0;
    if (lane == 0) c0 = (int32_t)atomicAdd(next_chunk, (unsigned)kCachedGrab);
    c0 = __shfl_sync(0xffffffffu, c0, 0) + c_begin;
    if (c0 >= c_end) break;
    const int32_t c1 = c0 + kCachedGrab < c_end ? c0 + kCachedGrab : c_end;
    if (lane < c1 - c0) {  // lane u prefetches chunk c0 + u (1 KB of colf)
      const int32_t cu = c0 + lane;
      int su = s;
      while (cu >= (int32_t)seg_chunk[su + 1]) ++su;
      prefetch_l2(colf + seg_cstart[su] + (int64_t)(cu - (int32_t)seg_chunk[su]) * kCachedChunk,
                  kCachedChunk * 4);
    }
    for (int32_t c = c0; c < c1; ++c) {
      if (c >= cnext) {
        while (c >= (int32_t)seg_chunk[s + 1]) ++s;
        lo = seg_lo[s];
        Es = seg_E[s];
        cstart = (int32_t)seg_cstart[s];
        cbase = (int32_t)seg_chunk[s];
        cnext = (int32_t)seg_chunk[s + 1];
      }
      cached_chunk<Op>(colf, x, nx, lo, Es, cstart, c - cbase, c, first_row[c], out, carry);
    }
  }
}

// Both kinds in one launch (one 1024-thread block per SM): threads
// [0, staged_threads) run the staged schedule (named barrier 1 among them),
// the other warps serve the L1/L2 segments from the chunk queue from the
// start, and the staged warps join that queue when their pieces run out.
// The cold segments' random reads go to L2 while the staged warps read
// shared memory, so the two kinds of lookup proceed side by side.
template <class Op>
__global__ void __launch_bounds__(1024, 1)
overlap_gather_kernel(const uint8_t* __restrict__ cs, const uint32_t* __restrict__ colf,
                      const typename Op::T* __restrict__ x, int32_t nx,
                      const int32_t* __restrict__ first_row,
                      const int64_t* __restrict__ seg_cstart, const int32_t* __restrict__ seg_E,
                      const int64_t* __restrict__ seg_chunk,
                      const int32_t* __restrict__ seg_ctile, const int32_t* __restrict__ seg_lo,
                      const int32_t* __restrict__ seg_tab, int m, int k, int32_t ct_end,
                      int32_t piece, int staged_threads, unsigned* __restrict__ counters,
                      typename Op::T* __restrict__ out, typename Op::T* __restrict__ carry) {
  using T = typename Op::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int32_t s_piece, s_size;
  if ((int)threadIdx.x < staged_threads)
    staged_pieces<Op>(cs, x, seg_E, seg_chunk, seg_ctile, seg_lo, seg_tab, ct_end, piece,
                      counters, out, carry, reinterpret_cast<T*>(smem_raw), staged_threads,
                      &s_piece, &s_size);
  cached_queue<Op>(colf, x, nx, first_row, seg_cstart, seg_E, seg_chunk, seg_lo, m, k,
                   counters + 1, out, carry);
}

}  // namespace

int seg_table_capacity(int ctas) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  int sm_smem = 0, reserved = 0, optin = 0;
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ctas < 1) ctas = 1;
  int64_t per = (int64_t)sm_smem / ctas - reserved;
  if (per > optin) per = optin;
  per -= 128;  // the gather kernels' own static shared memory
  if (per <= 0) return 0;
  return (int)((per / 4) & ~31LL);
}

int seg_plan_build(const int32_t* col, const int64_t* rp, const int32_t* rp32, int64_t rows,
                   int64_t E, int k, const std::vector<int64_t>& row_base,
                   const std::vector<int64_t>& edge_base, const std::vector<int64_t>& src_bounds,
                   SegPlan* p, cudaStream_t s) {
  p->k = k;
  p->E = E;
  p->rows = rows;
  p->rp32 = rp32;
  p->row_base = row_base;
  p->edge_base = edge_base;
  p->src_bounds = src_bounds;
  p->h_cstart.assign(k + 1, 0);
  for (int q = 0; q < k; ++q) {
    const int64_t Eq = edge_base[q + 1] - edge_base[q];
    p->h_cstart[q + 1] = p->h_cstart[q] + ((Eq + 7) & ~7LL);
  }
  p->colf_len = p->h_cstart[k] + kMaxChunkEdges;  // chunks may read past their segment's end
  if (p->colf_len >= 0x7FFFFFFFLL) {
    set_error("segmented gather: padded edge array exceeds 2^31 entries");
    return CG_ERR_UNSUPPORTED;
  }
  CG_CUDA(cudaMalloc((void**)&p->colf, sizeof(uint32_t) * p->colf_len));
  CG_CUDA(cudaMemsetAsync(p->colf, 0, sizeof(uint32_t) * p->colf_len, s));
  const size_t kk = (size_t)(k > 0 ? k : 1);
  CG_CUDA(cudaMalloc((void**)&p->seg_cstart, sizeof(int64_t) * kk));
  CG_CUDA(cudaMalloc((void**)&p->seg_E, sizeof(int32_t) * kk));
  CG_CUDA(cudaMalloc((void**)&p->seg_chunk, sizeof(int64_t) * (kk + 1)));
  CG_CUDA(cudaMalloc((void**)&p->seg_ctile, sizeof(int32_t) * (kk + 1)));
  CG_CUDA(cudaMalloc((void**)&p->seg_lo, sizeof(int32_t) * kk));
  CG_CUDA(cudaMalloc((void**)&p->seg_tab, sizeof(int32_t) * kk));
  CG_CUDA(cudaMalloc((void**)&p->meta, sizeof(int64_t) * 4 * (kk + 1)));

  std::vector<int32_t> segE(kk, 0), lo(kk, 0);
  for (int q = 0; q < k; ++q) {
    segE[q] = (int32_t)(edge_base[q + 1] - edge_base[q]);
    lo[q] = (int32_t)src_bounds[q];
  }
  CG_CUDA(cudaMemcpyAsync(p->seg_cstart, p->h_cstart.data(), sizeof(int64_t) * k,
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(p->seg_E, segE.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(p->seg_lo, lo.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
  // meta: row_base, edge_base, cstart, bounds (k+1 each), for chunk indexing and export
  CG_CUDA(cudaMemcpyAsync(p->meta, row_base.data(), sizeof(int64_t) * (k + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(p->meta + (k + 1), edge_base.data(), sizeof(int64_t) * (k + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(p->meta + 2 * (k + 1), p->h_cstart.data(), sizeof(int64_t) * (k + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(p->meta + 3 * (k + 1), src_bounds.data(), sizeof(int64_t) * (k + 1),
                          cudaMemcpyHostToDevice, s));
  if (rows > 0) {
    colf_fill_kernel<<<grid_for(rows * 32, 256, 16), 256, 0, s>>>(
        col, rp, rows, p->meta, p->meta + (k + 1), p->meta + 2 * (k + 1), p->meta + 3 * (k + 1),
        k, p->colf);
    CG_LAUNCH_CHECK();
  }
  CG_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope
  return seg_plan_configure(p, 1024, 1, -1, s);
}

int seg_plan_configure(SegPlan* p, int threads, int ctas_per_sm, int tab_vertices,
                       cudaStream_t s) {
  if (threads != 512 && threads != 1024) {
    set_error("gather threads must be 512 or 1024 (got %d)", threads);
    return CG_ERR_INVALID_ARG;
  }
  const int max_ctas = 1024 / threads;  // the staged kernel holds 64 registers per thread
  if (ctas_per_sm < 1 || ctas_per_sm > max_ctas) {
    set_error("ctas_per_sm must be in [1, %d] for %d threads", max_ctas, threads);
    return CG_ERR_INVALID_ARG;
  }
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  const int cap = seg_table_capacity(ctas_per_sm);
  int tab = tab_vertices < 0 ? cap : std::min(tab_vertices, cap);
  tab = std::min(tab, 65536) & ~3;  // staged sources are 16-bit segment-local indices
  const int k = p->k;
  // staged prefix: leading segments that fit the table and carry enough
  // edges (>= 4 per source) for staging them in shared memory to pay
  // (with the segment-affine plan: >= affine_head edges per source, the
  // rest of the table-sized segments go one block per segment)
  const double head_deg = p->affine_head > 0.0 ? std::max(4.0, p->affine_head) : 4.0;
  int m = 0;
  int64_t tabmax = 0;
  while (m < k && tab > 0) {
    const int64_t size = p->src_bounds[m + 1] - p->src_bounds[m];
    const int64_t Eq = p->edge_base[m + 1] - p->edge_base[m];
    if (size > tab || (double)Eq < head_deg * (double)size) break;
    tabmax = std::max(tabmax, size);
    ++m;
  }
  // segment-affine staged segments [m, m2): the table-sized segments after the
  // head, when asked for (each one's table is staged once, by one block)
  int m2 = m;
  if (p->affine_head > 0.0) {
    if (threads != 1024 || ctas_per_sm != 1) {
      set_error("segment-affine staging needs 1024 threads and 1 block per SM (got %d x %d)",
                threads, ctas_per_sm);
      return CG_ERR_INVALID_ARG;
    }
    if (p->overlap_request > 0) {
      set_error("segment-affine staging and the overlapped gather exclude each other");
      return CG_ERR_INVALID_ARG;
    }
    while (m2 < k && tab > 0 && p->src_bounds[m2 + 1] - p->src_bounds[m2] <= tab) {
      tabmax = std::max(tabmax, p->src_bounds[m2 + 1] - p->src_bounds[m2]);
      ++m2;
    }
  }
  // one overlapped launch needs both kinds of segment and the 1024 x 1 shape
  bool cached_edges = false;
  for (int q = m2; q < k; ++q) cached_edges |= p->edge_base[q + 1] > p->edge_base[q];
  if (p->overlap_request > 0 && (threads != 1024 || ctas_per_sm != 1)) {
    set_error("gather overlap needs 1024 threads and 1 block per SM (got %d x %d)", threads,
              ctas_per_sm);
    return CG_ERR_INVALID_ARG;
  }
  p->overlap = (m > 0 && cached_edges) ? p->overlap_request : 0;
  const int chunk_a = kStagedChunk, chunk_b = kCachedChunk;
  const int warps_a = p->overlap > 0 ? 32 - p->overlap : threads / 32, warps_b = 1024 / 32;
  std::vector<int64_t> chunk(k + 1, 0);
  std::vector<int32_t> ctile(k + 1, 0), tn(k > 0 ? k : 1, 0);
  for (int q = 0; q < k; ++q) {
    const int64_t Eq = p->edge_base[q + 1] - p->edge_base[q];
    const int64_t nch = ceil_div(Eq, q < m2 ? chunk_a : chunk_b);
    chunk[q + 1] = chunk[q] + nch;
    // block-groups of the sweeping launches (none for the segment-affine segments)
    ctile[q + 1] = ctile[q] + (q < m ? (int32_t)ceil_div(nch, warps_a)
                                     : q < m2 ? 0 : (int32_t)ceil_div(nch, warps_b));
    tn[q] = q < m2 ? (int32_t)(p->src_bounds[q + 1] - p->src_bounds[q]) : 0;
  }
  const int64_t nchunks = chunk[k];
  if (nchunks > p->chunk_cap) {
    cudaFree(p->first_row);
    cudaFree(p->carry);
    p->first_row = nullptr;
    p->carry = nullptr;
    p->chunk_cap = 0;
    const size_t nc = (size_t)(nchunks > 0 ? nchunks : 1);
    CG_CUDA(cudaMalloc((void**)&p->first_row, sizeof(int32_t) * nc));
    CG_CUDA(cudaMalloc(&p->carry, sizeof(int32_t) * nc));
    p->chunk_cap = nchunks;
  }
  const int64_t cs_bytes = chunk[m2] * kStagedChunkBytes;
  if (cs_bytes > p->cs_cap) {
    cudaFree(p->cs);
    p->cs = nullptr;
    p->cs_cap = 0;
    CG_CUDA(cudaMalloc((void**)&p->cs, (size_t)cs_bytes));
    p->cs_cap = cs_bytes;
  }
  CG_CUDA(cudaMemcpyAsync(p->seg_chunk, chunk.data(), sizeof(int64_t) * (k + 1),
                          cudaMemcpyHostToDevice, s));
  CG_CUDA(cudaMemcpyAsync(p->seg_ctile, ctile.data(), sizeof(int32_t) * (k + 1),
                          cudaMemcpyHostToDevice, s));
  if (k > 0)
    CG_CUDA(cudaMemcpyAsync(p->seg_tab, tn.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice,
                            s));
  if (nchunks > 0) {
    first_row_kernel<<<grid_for(nchunks, 256), 256, 0, s>>>(
        p->rp32, p->meta, p->meta + (k + 1), p->seg_chunk, k, m2, chunk_a, chunk_b, nchunks,
        p->first_row);
    CG_LAUNCH_CHECK();
  }
  if (chunk[m2] > 0) {
    staged_fill_kernel<<<grid_for(chunk[m2] * 32, 256), 256, 0, s>>>(
        p->colf, p->seg_chunk, p->seg_cstart, p->seg_E, p->first_row, m2, chunk[m2], p->cs);
    CG_LAUNCH_CHECK();
  }
  // static runs of carries, cut into pieces for the parallel completion
  cudaFree(p->fx_pieces);
  cudaFree(p->fx_runs);
  cudaFree(p->fx_sum);
  cudaFree(p->fx_done);
  p->fx_pieces = nullptr;
  p->fx_runs = nullptr;
  p->fx_sum = nullptr;
  p->fx_done = nullptr;
  p->fx_npieces = p->fx_nruns = 0;
  if (nchunks > 0) {
    int32_t* orow = nullptr;
    CG_CUDA(cudaMallocAsync((void**)&orow, sizeof(int32_t) * (size_t)nchunks, s));
    open_row_kernel<<<grid_for(nchunks, 256), 256, 0, s>>>(
        p->rp32, p->meta, p->meta + (k + 1), p->seg_chunk, k, m2, chunk_a, chunk_b, nchunks, orow);
    cudaError_t ce = cudaGetLastError();
    std::vector<int32_t> hc((size_t)nchunks);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(hc.data(), orow, sizeof(int32_t) * (size_t)nchunks,
                           cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFreeAsync(orow, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "segmented gather: carry runs", __FILE__, __LINE__);
    std::vector<int4> hp, hr;
    for (int64_t c = 0; c < nchunks;) {
      if (hc[c] < 0) { ++c; continue; }
      int64_t e = c + 1;
      while (e < nchunks && hc[e] == hc[c]) ++e;
      const int32_t run = (int32_t)hr.size(), p0 = (int32_t)hp.size();
      for (int64_t x = c; x < e; x += 32)
        hp.push_back(make_int4((int32_t)x, (int32_t)std::min<int64_t>(32, e - x), run, 0));
      hr.push_back(make_int4(hc[c], p0, (int32_t)hp.size() - p0, 0));
      c = e;
    }
    p->fx_npieces = (int64_t)hp.size();
    p->fx_nruns = (int64_t)hr.size();
    if (!hp.empty()) {
      CG_CUDA(cudaMalloc((void**)&p->fx_pieces, sizeof(int4) * hp.size()));
      CG_CUDA(cudaMalloc((void**)&p->fx_runs, sizeof(int4) * hr.size()));
      CG_CUDA(cudaMalloc(&p->fx_sum, 4 * hp.size()));
      CG_CUDA(cudaMalloc((void**)&p->fx_done, sizeof(unsigned) * hr.size()));
      CG_CUDA(cudaMemcpyAsync(p->fx_pieces, hp.data(), sizeof(int4) * hp.size(),
                              cudaMemcpyHostToDevice, s));
      CG_CUDA(cudaMemcpyAsync(p->fx_runs, hr.data(), sizeof(int4) * hr.size(),
                              cudaMemcpyHostToDevice, s));
      CG_CUDA(cudaMemsetAsync(p->fx_done, 0, sizeof(unsigned) * hr.size(), s));
    }
  }
  CG_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  p->threads = threads;
  p->ctas_per_sm = ctas_per_sm;
  p->tab_cap = (int)((tabmax + 3) & ~3LL);
  p->table_request = tab;
  p->m = m;
  p->m2 = m2;
  p->grid_affine = di.sm_count;
  p->nchunks = nchunks;
  p->ct_split = ctile[m];
  p->n_ctiles = ctile[k];
  p->grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(p->ct_split, (int64_t)di.sm_count * ctas_per_sm));
  if (p->overlap > 0) p->grid = di.sm_count;  // every SM serves the L1/L2 queue too
  // about eight pieces per block: balance without many table reloads
  p->piece = (int32_t)std::max<int64_t>(1, ceil_div(p->ct_split, 8LL * p->grid));
  if (!p->counter) CG_CUDA(cudaMalloc((void**)&p->counter, 3 * sizeof(unsigned)));
  p->grid_l2 = (int)std::max<int64_t>(
      1, std::min<int64_t>(p->n_ctiles - p->ct_split, (int64_t)di.sm_count * 2));
  return CG_OK;
}

void seg_plan_free(SegPlan* p) {
  cudaFree(p->counter);
  cudaFree(p->colf);
  cudaFree(p->cs);
  cudaFree(p->meta);
  cudaFree(p->seg_cstart);
  cudaFree(p->seg_E);
  cudaFree(p->seg_chunk);
  cudaFree(p->seg_ctile);
  cudaFree(p->seg_lo);
  cudaFree(p->seg_tab);
  cudaFree(p->first_row);
  cudaFree(p->carry);
  cudaFree(p->fx_pieces);
  cudaFree(p->fx_runs);
  cudaFree(p->fx_sum);
  cudaFree(p->fx_done);
  *p = SegPlan();
}

int64_t seg_plan_bytes(const SegPlan& p) {
  return 4 * p.colf_len + p.cs_cap + 8 * p.chunk_cap + 72 * (int64_t)p.k + 20 * p.fx_npieces +
         20 * p.fx_nruns;
}

int seg_plan_export_col(const SegPlan& p, const int32_t* rp, int32_t* col, cudaStream_t s) {
  if (p.rows == 0) return CG_OK;
  const int k = p.k;
  export_col_kernel<<<grid_for(p.rows * 32, 256, 16), 256, 0, s>>>(
      p.colf, rp, p.rows, p.meta, p.meta + (k + 1), p.meta + 2 * (k + 1), p.meta + 3 * (k + 1), k,
      col);
  CG_LAUNCH_CHECK();
  CG_CUDA(cudaStreamSynchronize(s));
  return CG_OK;
}

template <class Op, int THREADS>
static int launch_staged(const SegPlan& p, const typename Op::T* x, typename Op::T* out,
                         cudaStream_t s) {
  using T = typename Op::T;
  const size_t smem = (size_t)p.tab_cap * sizeof(T);
  auto fn = staged_gather_kernel<Op, THREADS>;
  CG_CUDA(cudaMemsetAsync(p.counter, 0, sizeof(unsigned), s));
  if (smem > 48 * 1024)
    CG_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  fn<<<p.grid, THREADS, smem, s>>>(p.cs, x, p.seg_E, p.seg_chunk, p.seg_ctile, p.seg_lo,
                                   p.seg_tab, p.ct_split, p.piece, p.counter, out,
                                   reinterpret_cast<T*>(p.carry));
  CG_LAUNCH_CHECK();
  return CG_OK;
}

template <class Op>
static int launch_overlap(const SegPlan& p, const typename Op::T* x, int32_t nx,
                          typename Op::T* out, cudaStream_t s) {
  using T = typename Op::T;
  const size_t smem = (size_t)p.tab_cap * sizeof(T);
  auto fn = overlap_gather_kernel<Op>;
  CG_CUDA(cudaMemsetAsync(p.counter, 0, 2 * sizeof(unsigned), s));
  if (smem > 48 * 1024)
    CG_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  fn<<<p.grid, 1024, smem, s>>>(p.cs, p.colf, x, nx, p.first_row, p.seg_cstart, p.seg_E,
                                p.seg_chunk, p.seg_ctile, p.seg_lo, p.seg_tab, p.m, p.k,
                                p.ct_split, p.piece, 1024 - 32 * p.overlap, p.counter, out,
                                reinterpret_cast<T*>(p.carry));
  CG_LAUNCH_CHECK();
  return CG_OK;
}

template <class Op>
int run_seg_gather(const SegPlan& p, const typename Op::T* x, int32_t nx, typename Op::T* out,
                   cudaStream_t s, int phases) {
  if (p.nchunks == 0) return CG_OK;
  using T = typename Op::T;
  if (p.overlap > 0) {  // both kinds in one launch, counted as the staged phase
    if (phases & kPhaseStaged) CG_TRY((launch_overlap<Op>(p, x, nx, out, s)));
    phases &= ~(kPhaseStaged | kPhaseCached);
  }
  // staged segments [0, m): read from a shared-memory copy
  if ((phases & kPhaseStaged) && p.m > 0 && p.ct_split > 0) {
    if (p.threads == 1024)
      CG_TRY((launch_staged<Op, 1024>(p, x, out, s)));
    else
      CG_TRY((launch_staged<Op, 512>(p, x, out, s)));
  }
  // the table-sized cold segments, one block per segment
  if ((phases & kPhaseCached) && p.m2 > p.m) {
    const size_t smem = (size_t)p.tab_cap * sizeof(T);
    auto fn = affine_gather_kernel<Op>;
    CG_CUDA(cudaMemsetAsync(p.counter + 2, 0, sizeof(unsigned), s));
    if (smem > 48 * 1024)
      CG_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    fn<<<p.grid_affine, 1024, smem, s>>>(p.cs, x, p.seg_E, p.seg_chunk, p.seg_lo, p.seg_tab, p.m,
                                         p.m2, p.counter + 2, out, reinterpret_cast<T*>(p.carry));
    CG_LAUNCH_CHECK();
  }
  // the rest through L1/L2: no shared memory, so the whole on-chip store is L1
  if ((phases & kPhaseCached) && p.n_ctiles > p.ct_split) {
    seg_gather_kernel<Op, 1024><<<p.grid_l2, 1024, 0, s>>>(
        p.colf, x, nx, p.first_row, p.seg_cstart, p.seg_E, p.seg_chunk, p.seg_ctile, p.seg_lo,
        p.k, p.ct_split, (int32_t)p.n_ctiles, out, reinterpret_cast<T*>(p.carry));
    CG_LAUNCH_CHECK();
  }
  if ((phases & kPhaseFixup) && p.fx_npieces > 0) {
    seg_fixup_kernel<Op><<<grid_for(p.fx_npieces, 256, 4), 256, 0, s>>>(
        p.fx_pieces, p.fx_npieces, p.fx_runs, reinterpret_cast<const T*>(p.carry),
        reinterpret_cast<T*>(p.fx_sum), p.fx_done, out);
    CG_LAUNCH_CHECK();
  }
  return CG_OK;
}

template int run_seg_gather<SumF32>(const SegPlan&, const float*, int32_t, float*, cudaStream_t,
                                    int);
template int run_seg_gather<MinI32>(const SegPlan&, const int32_t*, int32_t, int32_t*,
                                    cudaStream_t, int);

}  // namespace cg
