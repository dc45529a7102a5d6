// Dense hub block of the batched personalised PageRank on the 5th-generation
// tensor cores (tcgen05).
//
// After frequency-based clustering (Section V) the hottest vertices carry the
// lowest IDs, and the block of the adjacency matrix among the first h of them
// is dense (on RMAT-22, the 16,384 x 16,384 hub block holds 15% of the edges
// at 3.7% density).  For those edges the gather of Algorithm 3 costs a
// 256-byte row read each, while a dense multiply costs a few FLOPs per matrix
// entry: the hub block becomes a contraction
//     Y[v][j] = sum_{u < h, u -> v} C[u][j]       for the destinations v < h,
// i.e. Y = A_H C_H with A_H the 0/1 hub block (row = destination) and C_H the
// hubs' contributions (64 columns, BF16 hi and lo planes).  Y is one more
// intermBuf row per hub destination, summed by the merge like any other row;
// the hub-block edges are removed from the segmented graph the gather walks
// (cg_split_hub_block).
//
// Kernel (CTAs of 288 threads: eight expander warps and one MMA/copy warp;
// each 128-destination tile's chunk list split over `parts` CTAs, whose
// partial rows the tile's last CTA to finish adds in part order, so the merge
// sees one dense row per hub destination):
//   A tile  128 destinations x 64 sources, BF16 0/1, expanded into shared
//           memory from the chunk's 1 KB of bitmap by the expander warps (two
//           threads per destination row, a byte -> 8 BF16 lookup table), which
//           then arrive on the stage's bar_ready mbarrier;
//   B tiles 64 columns x 64 sources for the hi and the lo plane, pre-packed
//           in global memory in the operand layout (ppr_dense_pack, after each
//           merge); bitmap and B tiles arrive by three bulk TMA copies per
//           chunk, issued by one thread of the MMA/copy warp two chunks ahead
//           once the stage's earlier MMAs have completed;
//   MMA     tcgen05.mma.cta_group::1.kind::f16, M = 128, N = 64, K = 16, FP32
//           accumulators in tensor memory (64 columns), four K-steps per plane
//           per chunk, issued by that same thread when the stage is ready and
//           committed to the stage's bar_mma mbarrier;
//   stages  three shared-memory stages (two CTAs per SM): the copies of
//           chunks i+1 and i+2 are in flight while chunk i is expanded and the
//           tensor cores work on i-1; no block-wide barrier per chunk;
//   sparse  64-source chunks with no edge in a tile's rows are skipped (a
//           per-tile list built once);
//   out     tcgen05.ld of the accumulators (warp w: rows 32w..32w+31), stored
//           as the tile's 128 intermBuf rows.
// Operand layout (both K-major, no swizzle): 8 x 16-byte core matrices;
// element (row r, k) of a tile lies at (r/8)*1024 + (k/8)*128 + (r%8)*16 +
// (k%8)*2 bytes, so LBO (next core matrix along K) = 128 and SBO (next 8 rows)
// = 1024.  Products of 0/1 and BF16 values are exact; the FP32 accumulation is
// the only rounding.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "ppr.cuh"

namespace cg {
namespace {

constexpr int kDM = 128;                   // destinations per tile (MMA M)
constexpr int kDK = 64;                    // sources per chunk
constexpr int kTileA = kDM * kDK * 2;      // 16 KB
constexpr int kTileB = kCols * kDK * 2;    // 8 KB per plane
constexpr int kTileBits = kDM * kDK / 8;   // 1 KB of bitmap per tile chunk
constexpr int kStage = kTileA + 2 * kTileB + kTileBits;  // 33 KB
constexpr int kStages = 3;                 // shared-memory stages (two CTAs per SM fit)
constexpr int kAhead = 2;                  // chunks whose copies are issued ahead
constexpr int kDThreads = 256;             // expander threads per CTA: two per destination row
constexpr uint32_t kDenseWaitPolls = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Expect `bytes` on bar's current phase and copy them global -> shared (TMA,
// both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{ .reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Arrive on bar (release: this thread's earlier shared-memory writes are
// visible to a thread that sees the phase complete).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{ .reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Wait for the phase of parity ph; false after kDenseWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t ph) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < kDenseWaitPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(ph)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory matrix descriptor: start address, LBO, SBO (bytes, all
// multiples of 16), descriptor version 1 (bits 46-48 = 0b001), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulators (bits 4-5 = 1),
// BF16 A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kCols >> 3) << 17) |
                            ((uint32_t)(kDM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 lanes x 32 columns of FP32 accumulators into registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Byte offset of element (row r, k) in a K-major tile without swizzle.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// One CTA per (128 hub destinations, part of their chunk list): tile t =
// blockIdx.x / parts, part p = blockIdx.x % parts takes chunks
// [p n / parts, (p+1) n / parts) of the tile's n non-empty chunks and writes
// its partial rows to partial[p][128t ..]; the tile's last part to finish
// adds the parts in order into rows 128t .. of out_rows.
// bits_t: the bitmap tile-major, 1 KB (128 rows x 2 words) per (tile, chunk).
// Warp-specialised pipeline over the part's chunks i (stage i % 3), linked by
// mbarriers only (no block barrier per chunk):
//   warps 0-7 (256 threads, two per destination row) wait for chunk i's
//     copies (bar_load[s]), expand the A tile from the staged bitmap and arrive
//     on bar_ready[s] (one arrival per warp);
//   warp 8, one thread, waits for bar_ready[s], issues chunk i's 8 MMAs and
//     commits them to bar_mma[s]; then issues the copies of chunk i + 2
//     (bitmap, B hi, B lo) into the stage that chunk i - 1's MMAs read, once
//     those are done (bar_mma of chunk i - 1).
// The expanders run up to two chunks ahead of the tensor cores.
__global__ void __launch_bounds__(kDThreads + 32, 2)
dense_tile_kernel(const uint32_t* __restrict__ bits_t, int32_t h, int parts,
                  const int32_t* __restrict__ tile_off_list, const int32_t* __restrict__ chunks,
                  const uint8_t* __restrict__ ct_hi, const uint8_t* __restrict__ ct_lo,
                  float* __restrict__ partial, unsigned* __restrict__ done,
                  float* __restrict__ out_rows, unsigned* __restrict__ fault) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar_load[kStages], bar_ready[kStages], bar_mma[kStages];
  __shared__ uint32_t s_taddr;
  __shared__ uint4 s_lut[256];  // byte -> 8 BF16 values, 1.0 where the bit is set
  __shared__ bool s_last;
  __shared__ int s_ok;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const bool expander = tid < kDThreads;  // warps 0-7; warp 8 copies and issues the MMAs
  const int t = blockIdx.x / parts, part = blockIdx.x % parts;
  const int nall = tile_off_list[t + 1] - tile_off_list[t];
  const int c0 = tile_off_list[t] + (int)((int64_t)part * nall / parts);
  const int nch = tile_off_list[t] + (int)((int64_t)(part + 1) * nall / parts) - c0;
  const int nchunk = h / kDK;
  // epilogue: warp w < 8 holds TMEM lanes 32(w%4).. and columns 32(w/4)..
  const int erow = 32 * (w & 3) + lane, ecol = 32 * ((w >> 2) & 1);
  const int64_t dst = (int64_t)t * kDM + erow;  // hub destination of this thread's half row
  float4* prow = reinterpret_cast<float4*>(partial + ((int64_t)part * h + dst) * kCols + ecol);
  // the tile's parts: each stores its partial rows; the last part to finish
  // (an atomic count, no waiting) adds them in part order into the output
  auto finish = [&]() {
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(done + t, 1u) == (unsigned)parts - 1;
    __syncthreads();
    if (!s_last || !expander) return;
    __threadfence();
    float4 acc[8];
    for (int q = 0; q < 8; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pp = 0; pp < parts; ++pp) {
      const float4* src = reinterpret_cast<const float4*>(partial + ((int64_t)pp * h + dst) * kCols + ecol);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 x = __ldcg(src + q);
        acc[q].x += x.x; acc[q].y += x.y; acc[q].z += x.z; acc[q].w += x.w;
      }
    }
    float4* orow = reinterpret_cast<float4*>(out_rows + dst * kCols + ecol);
#pragma unroll
    for (int q = 0; q < 8; ++q) orow[q] = acc[q];
    if (tid == 0) done[t] = 0u;  // ready for the next launch
  };
  if (nch == 0) {  // no hub-block edge for this part
    if (expander)
#pragma unroll
      for (int q = 0; q < 8; ++q) prow[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    finish();
    return;
  }
  if (expander) {
    uint32_t p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      p[q] = (((tid >> (2 * q)) & 1) ? 0x3F80u : 0u) | (((tid >> (2 * q + 1)) & 1) ? 0x3F800000u : 0u);
    s_lut[tid] = make_uint4(p[0], p[1], p[2], p[3]);
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&bar_load[q], 1);
      mbar_init(&bar_ready[q], kDThreads / 32);
      mbar_init(&bar_mma[q], 1);
    }
    fence_mbar_init();
    s_ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  bool ok = true;
  if (expander) {
    for (int i = 0; i < nch; ++i) {
      const int s = i % kStages;
      uint8_t* A = sm + s * kStage;
      const uint32_t* Bt = reinterpret_cast<const uint32_t*>(A + kTileA + 2 * kTileB);
      // chunk i's copies landed (they were issued after the MMAs of chunk
      // i - kStages, the last readers of this stage's A tile, were done)
      if (!mbar_wait(&bar_load[s], (i / kStages) & 1)) {
        ok = false;
        break;
      }
      {  // thread t: row t/2, sources 32(t%2) .. 32(t%2)+31 (one bitmap word)
        const int r = tid >> 1, hw = tid & 1;
        const uint32_t word = Bt[2 * r + hw];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(A + tile_off(r, 32 * hw + 8 * q)) = s_lut[(word >> (8 * q)) & 0xFFu];
      }
      fence_proxy_async_smem();  // the generic-proxy writes, before the MMAs read them
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_ready[s]);
    }
  } else if (lane == 0) {  // warp 8: copies and MMAs
    auto issue = [&](int j) {  // the copies of chunk j into stage j % kStages
      uint8_t* st = sm + (j % kStages) * kStage;
      uint64_t* bl = &bar_load[j % kStages];
      const int c = chunks[c0 + j];
      bulk_expect(bl, 2 * kTileB + kTileBits);
      bulk_copy(st + kTileA, ct_hi + (int64_t)c * kTileB, kTileB, bl);
      bulk_copy(st + kTileA + kTileB, ct_lo + (int64_t)c * kTileB, kTileB, bl);
      bulk_copy(st + kTileA + 2 * kTileB,
                reinterpret_cast<const uint8_t*>(bits_t) + ((int64_t)t * nchunk + c) * kTileBits,
                kTileBits, bl);
    };
    for (int j = 0; j < kAhead && j < nch; ++j) issue(j);
    for (int i = 0; i < nch; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(&bar_ready[s], (i / kStages) & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint8_t* A = sm + s * kStage;
      const uint32_t a0 = smem_u32(A), h0 = smem_u32(A + kTileA), l0 = smem_u32(A + kTileA + kTileB);
#pragma unroll
      for (int kk = 0; kk < kDK / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
        mma_bf16(taddr, ad, smem_desc(h0 + kk * 256, 128, 1024), (i > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(taddr, ad, smem_desc(l0 + kk * 256, 128, 1024), 1u);
      }
      mma_commit(&bar_mma[s]);  // arrives once this thread's MMAs so far have completed
      const int j = i + kAhead;
      if (j < nch) {
        // stage j % kStages was last read by the MMAs of chunk j - kStages
        const int old = j - kStages;
        if (old >= 0 && !mbar_wait(&bar_mma[old % kStages], (old / kStages) & 1)) {
          ok = false;
          break;
        }
        issue(j);
      }
    }
  }
  // the last chunk's commit covers every MMA issued before it; a thread that
  // gave up waiting stops the others' epilogue through s_ok
  if (!ok) atomicAnd(&s_ok, 0);
  const int last = nch - 1;
  if (ok && expander && !mbar_wait(&bar_mma[last % kStages], (last / kStages) & 1))
    atomicAnd(&s_ok, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  ok = s_ok != 0;
  if (ok && expander) {
    float v[32];
    tmem_ld32(taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)ecol, v);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      prow[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if (!ok && tid == 0) {
    atomicOr(fault, 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(kCols)
                 : "memory");
  }
  finish();
}

// The bitmap tile-major: for tile t and chunk c, 128 rows x 2 words.
__global__ void dense_tile_bits_kernel(const uint32_t* __restrict__ bits, int32_t h,
                                       uint32_t* __restrict__ bits_t) {
  const int wpr = h >> 5, nchunk = h / kDK;
  const int64_t total = (int64_t)h * wpr;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = x / wpr;
    const int wd = (int)(x % wpr);
    const int64_t t = v / kDM;
    const int r = (int)(v % kDM), c = wd >> 1;
    bits_t[((t * nchunk + c) * kDM + r) * 2 + (wd & 1)] = bits[x];
  }
}

// The hubs' contributions in the B operand layout: chunk c = u / 64 holds
// 64 columns x 64 sources; column n of source u at tile_off(n, u % 64).
__global__ void dense_pack_kernel(const uint4* __restrict__ c_hi, const uint4* __restrict__ c_lo,
                                  int32_t h, uint8_t* __restrict__ ct_hi,
                                  uint8_t* __restrict__ ct_lo) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)h * 8;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = x >> 3;
    const int g = (int)(x & 7);  // columns 8g .. 8g+7
    const int k = (int)(u & (kDK - 1));
    uint8_t* dh = ct_hi + (u / kDK) * kTileB;
    uint8_t* dl = ct_lo + (u / kDK) * kTileB;
    const uint4 a = c_hi[u * 8 + g];
    const uint4 b = c_lo ? c_lo[u * 8 + g] : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t o = tile_off(8 * g + q, k);
      *reinterpret_cast<uint16_t*>(dh + o) = (uint16_t)(wa[q >> 1] >> (16 * (q & 1)));
      *reinterpret_cast<uint16_t*>(dl + o) = (uint16_t)(wb[q >> 1] >> (16 * (q & 1)));
    }
  }
}

// Which 64-source chunks of each 128-destination tile hold an edge.
__global__ void dense_chunk_flags_kernel(const uint32_t* __restrict__ bits, int32_t h,
                                         uint8_t* __restrict__ flags) {
  const int nchunk = h / kDK, wpr = h >> 5;
  const int64_t total = (int64_t)(h / kDM) * nchunk;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = x / nchunk;
    const int c = (int)(x % nchunk);
    uint32_t any = 0;
    for (int r = 0; r < kDM; ++r) {
      const uint32_t* wr = bits + (t * kDM + r) * wpr + (int64_t)c * 2;
      any |= wr[0] | wr[1];
    }
    flags[x] = any != 0;
  }
}

// Destination-major row lists with `parts` more rows (the dense partial rows,
// part order) at the end of each hub destination's list.
__global__ void dense_rows_kernel(const int32_t* __restrict__ old_off,
                                  const int32_t* __restrict__ old_rows, int32_t V, int32_t h,
                                  int parts, int64_t rows0, int32_t* __restrict__ new_off,
                                  int32_t* __restrict__ new_rows) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t extra = (int32_t)(v < h ? v : h) * parts;
    new_off[v] = old_off[v] + extra;
    if (v == V) continue;
    const int32_t b = old_off[v], e = old_off[v + 1], nb = b + extra;
    for (int32_t i = b; i < e; ++i) new_rows[nb + (i - b)] = old_rows[i];
    if (v < h)
      for (int q = 0; q < parts; ++q)
        new_rows[nb + (e - b) + q] = (int32_t)(rows0 + (int64_t)q * h + v);
  }
}

// ---- the hub-block split of an in-edge CSR
__global__ void split_count_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                                   int32_t V, int32_t h, int32_t* __restrict__ keep,
                                   uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int wpr = h >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nw) {
    int32_t k = 0;
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) {
      const int32_t u = src[e];
      if (v < h && u < h)
        atomicOr(bits + v * wpr + (u >> 5), 1u << (u & 31));
      else
        ++k;
    }
    k = warp_sum(k);
    if (lane == 0) keep[v] = k;
  }
}

__global__ void split_copy_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                                  int32_t V, int32_t h, const int64_t* __restrict__ out_off,
                                  int32_t* __restrict__ out_src) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += nw) {
    int64_t o = out_off[v];
    for (int64_t e0 = off[v]; e0 < off[v + 1]; e0 += 32) {
      const int64_t e = e0 + lane;
      int32_t u = 0;
      bool kp = false;
      if (e < off[v + 1]) {
        u = src[e];
        kp = !(v < h && u < h);
      }
      const unsigned m = __ballot_sync(0xffffffffu, kp);
      if (kp) out_src[o + __popc(m & ((1u << lane) - 1u))] = u;
      o += __popc(m);
    }
  }
}

}  // namespace

int ppr_dense_launch(cg_ppr* p, cudaStream_t s) {
  if (p->dense_h == 0) return CG_OK;
  if (p->dense_fault && *(volatile unsigned*)p->dense_fault) {
    *(volatile unsigned*)p->dense_fault = 0u;
    set_error("batched PPR: a dense-tile launch gave up waiting on its copies or its "
              "tensor-core work (its rows are incomplete)");
    return CG_ERR_TIMEOUT;
  }
  const int smem = kStages * kStage;
  CG_CUDA(cudaFuncSetAttribute((const void*)dense_tile_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  dense_tile_kernel<<<(p->dense_h / kDM) * p->dense_parts, kDThreads + 32, smem, s>>>(
      p->dense_bits_t, p->dense_h, p->dense_parts, p->dense_tile_off, p->dense_tile_chunks,
      p->ct_hi, p->ct_lo, p->dense_partial, p->dense_done, p->interm + p->dense_rows0 * kCols,
      p->dense_fault_dev);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

int ppr_dense_pack(cg_ppr* p, cudaStream_t s) {
  if (p->dense_h == 0) return CG_OK;
  dense_pack_kernel<<<grid_for((int64_t)p->dense_h * 8, 256), 256, 0, s>>>(
      p->c_hi, p->c_lo, p->dense_h, p->ct_hi, p->ct_lo);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

void ppr_dense_free(cg_ppr* p) {
  cudaFree(p->dense_tile_off);
  cudaFree(p->dense_tile_chunks);
  cudaFree(p->ct_hi);
  cudaFree(p->ct_lo);
  cudaFree(p->dense_bits_t);
  cudaFree(p->dense_partial);
  cudaFree(p->dense_done);
  p->dense_bits_t = nullptr;
  p->dense_partial = nullptr;
  p->dense_done = nullptr;
  if (p->dense_fault) cudaFreeHost(p->dense_fault);
  p->dense_tile_off = p->dense_tile_chunks = nullptr;
  p->ct_hi = p->ct_lo = nullptr;
  p->dense_fault = p->dense_fault_dev = nullptr;
}

}  // namespace cg

using namespace cg;

extern "C" {

int cg_split_hub_block(const int64_t* in_offsets, const int32_t* in_src, int32_t V, int64_t E,
                       int32_t h, int64_t* out_offsets, int32_t* out_src, uint32_t* dev_bits,
                       int64_t* E_rest, cudaStream_t stream) {
  CG_ARG(V >= 1 && E >= 0 && E < 0x7FFFFFFFLL, "cg_split_hub_block: V >= 1 and 0 <= E < 2^31-1");
  CG_ARG(h >= kDM && h % kDM == 0 && h <= V,
         "cg_split_hub_block: h must be a positive multiple of %d and <= V (got %d)", kDM, h);
  CG_ARG(in_offsets && out_offsets && dev_bits && E_rest && (E == 0 || (in_src && out_src)),
         "cg_split_hub_block: null pointer argument");
  CG_TRY(validate_csr(in_offsets, in_src, V, E, stream));
  int32_t* keep = nullptr;
  CG_CUDA(cudaMemsetAsync(dev_bits, 0, sizeof(uint32_t) * (size_t)h * (size_t)(h / 32), stream));
  cudaError_t e = cudaMallocAsync((void**)&keep, sizeof(int32_t) * (size_t)V, stream);
  int st = e == cudaSuccess ? CG_OK : cuda_fail(e, "cg_split_hub_block", __FILE__, __LINE__);
  if (st == CG_OK) {
    split_count_kernel<<<grid_for((int64_t)V * 32, 256), 256, 0, stream>>>(in_offsets, in_src, V,
                                                                           h, keep, dev_bits);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "cg_split_hub_block", __FILE__, __LINE__);
  }
  if (st == CG_OK) st = exclusive_scan_i32_to_i64(keep, out_offsets, V, stream);
  if (st == CG_OK) {
    split_copy_kernel<<<grid_for((int64_t)V * 32, 256), 256, 0, stream>>>(in_offsets, in_src, V,
                                                                          h, out_offsets, out_src);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(E_rest, out_offsets + V, sizeof(int64_t), cudaMemcpyDeviceToHost,
                          stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = cuda_fail(e, "cg_split_hub_block", __FILE__, __LINE__);
  }
  if (keep) cudaFreeAsync(keep, stream);
  return st;
}

int ppr_batched_attach_dense(cg_ppr* p, int32_t h, const uint32_t* dev_bits,
                             cudaStream_t stream) {
  CG_ARG(p != nullptr, "ppr_batched_attach_dense: null handle");
  CG_ARG(p->dense_h == 0, "ppr_batched_attach_dense: a dense block is attached already");
  CG_ARG(h >= kDM && h % kDM == 0 && h <= p->V,
         "ppr_batched_attach_dense: h must be a positive multiple of %d and <= V (got %d)", kDM,
         h);
  CG_ARG(dev_bits != nullptr, "ppr_batched_attach_dense: null bitmap");
  int cc_major = 0, cc_minor = 0, dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  CG_CUDA(cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev));
  CG_CUDA(cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
  if (cc_major != 10) {
    set_error("ppr_batched_attach_dense: tcgen05 needs a compute capability 10.x GPU (got %d.%d)",
              cc_major, cc_minor);
    return CG_ERR_UNSUPPORTED;
  }
  const int ntile = h / kDM, nchunk = h / kDK;
  // non-empty chunks per tile
  uint8_t* flags = nullptr;
  CG_CUDA(cudaMallocAsync((void**)&flags, (size_t)ntile * nchunk, stream));
  dense_chunk_flags_kernel<<<grid_for((int64_t)ntile * nchunk, 256), 256, 0, stream>>>(dev_bits, h,
                                                                                     flags);
  cudaError_t ce = cudaGetLastError();
  std::vector<uint8_t> hf((size_t)ntile * nchunk);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(hf.data(), flags, hf.size(), cudaMemcpyDeviceToHost, stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
  cudaFreeAsync(flags, stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "ppr_batched_attach_dense", __FILE__, __LINE__);
  std::vector<int32_t> toff(ntile + 1, 0), tch;
  for (int t = 0; t < ntile; ++t) {
    for (int c = 0; c < nchunk; ++c)
      if (hf[(size_t)t * nchunk + c]) tch.push_back(c);
    toff[t + 1] = (int32_t)tch.size();
  }
  if (tch.empty()) tch.push_back(0);
  int st = CG_OK;
  auto fail = [&](cudaError_t e) {
    ppr_dense_free(p);
    return cuda_fail(e, "ppr_batched_attach_dense", __FILE__, __LINE__);
  };
  cudaError_t e = cudaMalloc((void**)&p->dense_tile_off, sizeof(int32_t) * toff.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->dense_tile_chunks, sizeof(int32_t) * tch.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->ct_hi, (size_t)nchunk * kTileB);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->ct_lo, (size_t)nchunk * kTileB);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&p->dense_bits_t, sizeof(uint32_t) * (size_t)h * (size_t)(h / 32));
  if (e == cudaSuccess) {
    dense_tile_bits_kernel<<<grid_for((int64_t)h * (h / 32), 256), 256, 0, stream>>>(
        dev_bits, h, p->dense_bits_t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(p->ct_lo, 0, (size_t)nchunk * kTileB, stream);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&p->dense_fault, sizeof(unsigned), cudaHostAllocMapped);
  if (e == cudaSuccess) {
    *p->dense_fault = 0u;
    e = cudaHostGetDevicePointer((void**)&p->dense_fault_dev, p->dense_fault, 0);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->dense_tile_off, toff.data(), sizeof(int32_t) * toff.size(),
                        cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->dense_tile_chunks, tch.data(), sizeof(int32_t) * tch.size(),
                        cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return fail(e);
  // each tile's chunk list is split over `parts` CTAs (enough CTAs for every
  // SM), whose partial rows the tile's last CTA adds in part order: one more
  // intermBuf row per hub destination, listed last for it
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  const int parts = std::max(1, std::min(8, (2 * di.sm_count + ntile - 1) / ntile));
  e = cudaMalloc((void**)&p->dense_partial, sizeof(float) * kCols * (size_t)parts * (size_t)h);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->dense_done, sizeof(unsigned) * (size_t)ntile);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dense_done, 0, sizeof(unsigned) * (size_t)ntile, stream);
  if (e != cudaSuccess) return fail(e);
  int32_t *noff = nullptr, *nrows = nullptr;
  float* ninterm = nullptr;
  const int64_t rows2 = p->rows + h;
  e = cudaMalloc((void**)&noff, sizeof(int32_t) * ((size_t)p->V + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&nrows, sizeof(int32_t) * (size_t)rows2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ninterm, sizeof(float) * kCols * (size_t)rows2);
  if (e == cudaSuccess) {
    dense_rows_kernel<<<grid_for((int64_t)p->V + 1, 256), 256, 0, stream>>>(
        p->dst_off, p->dst_rows, p->V, h, 1, p->rows, noff, nrows);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaFree(noff);
    cudaFree(nrows);
    cudaFree(ninterm);
    return fail(e);
  }
  cudaFree(p->dst_off);
  cudaFree(p->dst_rows);
  cudaFree(p->interm);
  p->dst_off = noff;
  p->dst_rows = nrows;
  p->interm = ninterm;
  p->bytes += (int64_t)h * 4 + (int64_t)(parts + 1) * h * kCols * 4 + 4 * (int64_t)ntile +
              2 * (int64_t)nchunk * kTileB + 4 * (int64_t)(toff.size() + tch.size()) +
              (int64_t)h * (h / 8);
  p->dense_rows0 = p->rows;
  p->dense_parts = parts;
  p->dense_h = h;
  p->dense_bits = dev_bits;
  // the hubs' current contributions in the operand layout
  if (p->seeded) st = ppr_dense_pack(p, stream);
  return st;
}

}  // extern "C"
