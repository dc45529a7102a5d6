// Batched personalised PageRank handle (shared by ppr.cu and the dense-tile
// tensor-core path in ppr_dense.cu).
#pragma once

#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "handles.cuh"

namespace cg {

constexpr int kCols = 64;         // columns (rank vectors) per batch
constexpr int kChunk = 128;       // edges per octet chunk in the gather
constexpr int kTask = 16;         // destinations per octet task in the merge
constexpr int kThreads = 256;     // threads per block of every kernel here
constexpr uint32_t kRowEnd = 0x80000000u;

struct PprSeg {
  int64_t cstart;  // first flagged-edge entry of the segment
  int64_t chunk0;  // first gather chunk of the segment
  int32_t lo;      // first source vertex of the segment
  int32_t E;       // edges of the segment
};

}  // namespace cg

struct cg_ppr {
  int device = 0;
  const cg_segmented* seg = nullptr;
  int32_t V = 0;
  int32_t k = 0;
  int32_t planes = 2;
  int64_t rows = 0, nchunks = 0;
  cg::PprSeg* segs = nullptr;    // [k]
  int2* chunks = nullptr;        // [nchunks] (first subgraph row, segment)
  float* carry = nullptr;        // [nchunks][64]
  int4* pieces = nullptr;        // [npieces] (first chunk, chunks, run, -)
  int4* runs = nullptr;          // [nruns] (row, first piece, pieces, -)
  float* piece_sum = nullptr;    // [npieces][64]
  unsigned* run_done = nullptr;  // [nruns] pieces of the run finished (last-piece detection)
  int64_t npieces = 0, nruns = 0;
  int32_t* dst_off = nullptr;    // [V+1] destination-major row lists
  int32_t* dst_rows = nullptr;   // [rows]
  float* interm = nullptr;       // [rows][64] intermBuf
  uint4* c_hi = nullptr;         // [V][64] bf16
  uint4* c_lo = nullptr;         // [V][64] bf16 (two planes only)
  float* r_prev = nullptr;       // [V][64] R of the second-to-last iteration
  int32_t* seeds = nullptr;      // [64]
  uint32_t* seed_bits = nullptr; // [ceil(V/32)] vertices that are some column's seed
  double* D = nullptr;           // [64] dangling mass per column
  double* partials = nullptr;    // [merge_grid][128]
  unsigned* counter = nullptr;
  int merge_grid = 0, gather_grid = 0;
  bool seeded = false;
  int64_t bytes = 0;
  // dense hub block on the tensor cores (ppr_batched_attach_dense): the
  // edges among vertices [0, dense_h) of the graph are not in `seg` but in a
  // bitmap, multiplied by the hubs' contributions with tcgen05.mma
  int32_t dense_h = 0;               // 0: no dense block
  int32_t dense_parts = 1;           // CTAs (and dense rows) per 128-destination tile
  const uint32_t* dense_bits = nullptr;  // caller-owned [dense_h][dense_h/32]
  uint32_t* dense_bits_t = nullptr;  // the same bitmap tile-major (1 KB per tile chunk)
  float* dense_partial = nullptr;    // [dense_parts][dense_h][64] partial rows of the parts
  unsigned* dense_done = nullptr;    // [dense_h/128] parts finished per tile
  int32_t* dense_tile_off = nullptr;     // [dense_h/128 + 1] non-empty 64-source chunks per tile
  int32_t* dense_tile_chunks = nullptr;  // [total]
  uint8_t* ct_hi = nullptr;          // [dense_h/64][8192 B] hub contributions, MMA operand layout
  uint8_t* ct_lo = nullptr;
  int64_t dense_rows0 = 0;           // intermBuf row of hub destination 0's dense row
  unsigned* dense_fault = nullptr;   // host-mapped: a dense launch whose wait gave up
  unsigned* dense_fault_dev = nullptr;
};


namespace cg {
// The dense hub block (ppr_dense.cu): its tensor-core launch (after the
// sparse gather, before the merge), the packing of the hubs' contributions
// into the operand layout (after every merge and after init), and freeing.
int ppr_dense_launch(cg_ppr* p, cudaStream_t s);
int ppr_dense_pack(cg_ppr* p, cudaStream_t s);
void ppr_dense_free(cg_ppr* p);
}  // namespace cg
