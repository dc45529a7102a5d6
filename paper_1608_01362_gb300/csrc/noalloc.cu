// pr_iterate_plain_noalloc: one plain pull PageRank iteration that allocates
// nothing.  Some callers cannot allocate device memory at call time: code
// running under a fixed memory budget reserved up front, hosts embedding the
// library where only pre-registered buffers may be touched, or a caller that
// must not trigger the synchronisation an allocation can cause.  The plain
// path normally keeps its work buffers in a cg_plain handle; this variant
// keeps them instead in one statically sized device array in this file
// (every GPU that loads the library holds it until the process exits).
#include <mutex>

#include "gather.cuh"
#include "update.cuh"

namespace cg {
namespace {

constexpr int64_t kNoAllocMaxV = int64_t(1) << 20;  // vertices
constexpr int64_t kNoAllocMaxE = int64_t(1) << 24;  // edges
constexpr int64_t kNoAllocMaxTiles = (kNoAllocMaxV + kNoAllocMaxE + kTileItems - 1) / kTileItems;
constexpr int64_t kNoAllocMaxBlocks = (kNoAllocMaxV / 512 + kMergeWarps - 1) / kMergeWarps;

// Scratch layout (byte offsets, each 256-byte aligned).
constexpr int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }
constexpr int64_t kOffAcc = 0;                                               // float[V]
constexpr int64_t kOffTileRow = align256(kOffAcc + 4 * kNoAllocMaxV);        // int32[tiles+1]
constexpr int64_t kOffTileEdge = align256(kOffTileRow + 4 * (kNoAllocMaxTiles + 1));
constexpr int64_t kOffCarry = align256(kOffTileEdge + 4 * (kNoAllocMaxTiles + 1));  // float
constexpr int64_t kOffCarryRow = align256(kOffCarry + 4 * kNoAllocMaxTiles);       // int32
constexpr int64_t kOffPartials = align256(kOffCarryRow + 4 * kNoAllocMaxTiles);    // double
constexpr int64_t kOffCounter = align256(kOffPartials + 16 * kNoAllocMaxBlocks);   // unsigned
constexpr int64_t kScratchBytes = align256(kOffCounter + 4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device (with that
// device current).  In host code the array's name is only a host-side
// stand-in, so kernels get this address instead.
int scratch_address(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[64] = {nullptr};
  int dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return CG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    CG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = addr[dev];
  return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int pr_noalloc_limits(int64_t* max_vertices, int64_t* max_edges, int64_t* scratch_bytes) {
  if (max_vertices) *max_vertices = kNoAllocMaxV;
  if (max_edges) *max_edges = kNoAllocMaxE;
  if (scratch_bytes) *scratch_bytes = kScratchBytes;
  return CG_OK;
}

int pr_iterate_plain_noalloc(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E,
                             const float* inv, const float* rank_in, const float* contrib_in,
                             float* rank_out, float* contrib_out, double damping,
                             double* dangling_io, double* resid, cudaStream_t stream) {
  CG_ARG(V >= 1 && E >= 0, "pr_iterate_plain_noalloc: V must be >= 1 and E >= 0");
  CG_ARG(V <= kNoAllocMaxV, "pr_iterate_plain_noalloc: V = %d exceeds the fixed scratch limit "
         "of %lld vertices", V, (long long)kNoAllocMaxV);
  CG_ARG(E <= kNoAllocMaxE, "pr_iterate_plain_noalloc: E = %lld exceeds the fixed scratch "
         "limit of %lld edges", (long long)E, (long long)kNoAllocMaxE);
  CG_ARG(offsets && (E == 0 || src) && inv && rank_in && contrib_in && rank_out && contrib_out &&
             dangling_io,
         "pr_iterate_plain_noalloc: null pointer argument");
  CG_ARG(damping >= 0.0 && damping <= 1.0, "pr_iterate_plain_noalloc: damping must be in [0, 1]");
  CG_ARG(rank_out != rank_in && contrib_out != contrib_in && (const float*)rank_out != contrib_in &&
             (const float*)contrib_out != rank_in && rank_out != contrib_out,
         "pr_iterate_plain_noalloc: output vectors must not alias the inputs or each other");
  unsigned char* base = nullptr;
  CG_TRY(scratch_address(&base));
  float* acc = reinterpret_cast<float*>(base + kOffAcc);
  int32_t* tile_row = reinterpret_cast<int32_t*>(base + kOffTileRow);
  int32_t* tile_edge = reinterpret_cast<int32_t*>(base + kOffTileEdge);
  float* carry = reinterpret_cast<float*>(base + kOffCarry);
  int32_t* carry_row = reinterpret_cast<int32_t*>(base + kOffCarryRow);
  double* partials = reinterpret_cast<double*>(base + kOffPartials);
  unsigned* counter = reinterpret_cast<unsigned*>(base + kOffCounter);

  // the last-block counter must start at zero (a failed earlier call could
  // have left it set); the remaining scratch is fully overwritten below
  CG_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), stream));
  const int64_t ntiles = ceil_div((int64_t)V + E, kTileItems);
  tile_partition_kernel<int64_t><<<grid_for(ntiles + 1, 256), 256, 0, stream>>>(
      offsets + 1, V, E, kTileItems, ntiles, tile_row, tile_edge);
  CG_LAUNCH_CHECK();
  gather_tile_kernel<SumF32, kTileThreads, kTileIPT, false, int64_t>
      <<<(unsigned)ntiles, kTileThreads, 0, stream>>>(offsets + 1, src, contrib_in, V, tile_row,
                                                      tile_edge, acc, carry, carry_row);
  CG_LAUNCH_CHECK();
  carry_fixup_kernel<SumF32><<<grid_for(ntiles, 256, 4), 256, 0, stream>>>(carry, carry_row,
                                                                           ntiles, V, acc);
  CG_LAUNCH_CHECK();
  PrArgs a;
  a.inv = inv;
  a.rank_in = rank_in;
  a.rank_out = rank_out;
  a.contrib_out = contrib_out;
  a.base = (float)((1.0 - damping) / (double)V);
  a.d = (float)damping;
  a.inv_V = 1.0 / (double)V;
  a.D_in = dangling_io;
  a.D_out = dangling_io;
  a.resid_out = resid;
  a.partials = partials;
  a.counter = counter;
  a.V = V;
  a.seed = -1;
  const int B = 512;
  const int nb = (int)ceil_div(V, B);
  const size_t smem = (size_t)kMergeWarps * B * 4;
  dense_update_kernel<<<(unsigned)ceil_div(nb, kMergeWarps), kMergeWarps * 32, smem, stream>>>(
      acc, B, nb, a);
  CG_LAUNCH_CHECK();
  return CG_OK;
}

}  // extern "C"
