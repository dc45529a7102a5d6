// Segment processing (Algorithm 3) over the flattened segmented graph.
//
// Edge layout ("colf"): the subgraphs' source IDs, segment after segment,
// each segment starting on an 8-entry (32-byte) boundary; bit 31 of an entry
// marks the last edge of its subgraph row.  Every subgraph row has at least
// one edge, so row i is the (i+1)-th flagged edge: the gather needs no row
// pointers at all.
//
// Work unit: a warp owns a chunk of 32*IPL consecutive edges of one segment
// (IPL = 8, or 16 in the staged launch at one block per SM); lane l holds
// edges [IPL*l, IPL*l + IPL) of it (16-byte streaming loads).  Lanes
// fold their 8 values sequentially, emit every row that starts and ends
// inside them, and a warp-wide segmented scan over the lanes' open-row parts
// completes each lane's first row.  The row still open at the chunk's end
// goes to carry[chunk], folded in afterwards in chunk order.  No shared
// staging of edges and no block barriers between chunks.
//
// Two launches per pass.  The leading segments that fit an SM's shared
// memory (after clustering, the hot head: the paper's cache-sized segment,
// sized here to on-chip shared memory) are "staged": each block copies its
// current segment's source values into shared memory and every read of the
// segment is served from there.  The remaining segments are read through
// L1/L2 by a second launch that uses no shared memory, leaving the whole
// on-chip store to the L1 cache.  In both, a block owns a contiguous run of
// block-sized groups of chunks (so it meets at most a few segments and
// stages at most a few tables), in segment order.
#pragma once

#include <vector>

#include "gather.cuh"

namespace cg {

constexpr uint32_t kRowEndFlag = 0x80000000u;
constexpr int kMaxChunkEdges = 512;  // 32 lanes x 16 edges (staged launch, 1 block/SM)

struct SegPlan {
  int k = 0;
  int64_t E = 0, rows = 0, nchunks = 0;
  uint32_t* colf = nullptr;        // [colf_len] flagged, padded segment-local sources
  uint8_t* cs = nullptr;           // staged chunk stream (16-bit local indices + masks)
  int64_t cs_cap = 0;
  int64_t colf_len = 0;
  int64_t* seg_cstart = nullptr;   // [k]   first colf entry of each segment
  int32_t* seg_E = nullptr;        // [k]   edges of each segment
  int64_t* seg_chunk = nullptr;    // [k+1] first global chunk of each segment
  int32_t* seg_ctile = nullptr;    // [k+1] first block-group of each segment
  int32_t* seg_lo = nullptr;       // [k]   first source of each segment
  int32_t* seg_tab = nullptr;      // [k]   table entries used for each segment
  int32_t* first_row = nullptr;    // [nchunks] subgraph row of each chunk's first edge
  void* carry = nullptr;           // [nchunks] 4-byte values
  int64_t* meta = nullptr;         // [4(k+1)] row_base, edge_base, cstart, bounds (device)
  const int32_t* rp32 = nullptr;   // subgraph row starts (owned by the handle)
  int64_t chunk_cap = 0;           // capacity of first_row / carry
  std::vector<int64_t> h_cstart, src_bounds, edge_base, row_base;
  int threads = 1024;       // staged-segment launch shape
  int ctas_per_sm = 1;
  int tab_cap = 0;          // table entries of the staged launch (its largest segment)
  int table_request = 0;    // the capacity asked for
  int m = 0;                // segments [0, m) are staged in shared memory (all blocks sweep them)
  int m2 = 0;               // segments [m, m2): staged too, one block per segment (affine)
  double affine_head = 0.0;  // > 0: head threshold (edges per source) of the segment-affine
                            // plan; the table-sized segments after the head go one per block
  int grid_affine = 0;      // blocks of the segment-affine launch
  int32_t ct_split = 0;     // first block-group of the unstaged segments
  int64_t n_ctiles = 0;
  int grid = 0;             // staged launch blocks
  int32_t piece = 1;        // block-groups per work piece of the staged launch
  unsigned* counter = nullptr;  // [3] next staged work piece, next L1/L2 chunk (overlap),
                                //     next segment-affine segment
  int overlap_request = 0;  // warps per block given to the L1/L2 segments (0: two launches)
  int overlap = 0;          // the same, in effect (0 when one kind of segment is absent)
  int grid_l2 = 0;          // unstaged launch blocks (1024 threads, 2 per SM)
  // rows spanning chunks: runs of carries (a static structure) cut into
  // pieces of <= 32 chunks, completed in parallel (see run_seg_gather)
  int4* fx_pieces = nullptr;   // [fx_npieces] (first chunk, chunks, run, -)
  int4* fx_runs = nullptr;     // [fx_nruns] (row, first piece, pieces, -)
  void* fx_sum = nullptr;      // [fx_npieces] 4-byte piece sums
  unsigned* fx_done = nullptr; // [fx_nruns] finished pieces per run
  int64_t fx_npieces = 0, fx_nruns = 0;
};

// Largest shared table (entries, multiple of 32) for `ctas` blocks per SM.
int seg_table_capacity(int ctas);

// Build colf, the chunk index and the carry buffers from the unpadded
// segmented CSR (col[E] int32 global sources, rp[rows+1] int64 row starts;
// rp32: the same row starts in int32, kept by the handle).  Synchronizes.
int seg_plan_build(const int32_t* col, const int64_t* rp, const int32_t* rp32, int64_t rows,
                   int64_t E, int k, const std::vector<int64_t>& row_base,
                   const std::vector<int64_t>& edge_base, const std::vector<int64_t>& src_bounds,
                   SegPlan* p, cudaStream_t s);

// Launch shape: threads per block (512 or 1024), blocks per SM, table size
// (-1: the capacity; 0: none).  Synchronizes the stream.
int seg_plan_configure(SegPlan* p, int threads, int ctas_per_sm, int tab_vertices,
                       cudaStream_t s);

void seg_plan_free(SegPlan* p);
int64_t seg_plan_bytes(const SegPlan& p);

// Recover the unpadded source array (flags cleared) for export.
int seg_plan_export_col(const SegPlan& p, const int32_t* rp, int32_t* col, cudaStream_t s);

// Launch phases of one pass (all by default): the staged launch, the L1/L2
// launch (with the segment-affine staged launch before it, when configured)
// and the carry fix-up, in that order.  With the overlap in effect one
// launch serves both kinds of segment: it runs for kPhaseStaged and
// kPhaseCached launches nothing.
constexpr int kPhaseStaged = 1, kPhaseCached = 2, kPhaseFixup = 4, kPhaseAll = 7;

template <class Op>
int run_seg_gather(const SegPlan& p, const typename Op::T* x, int32_t nx, typename Op::T* out,
                   cudaStream_t s, int phases = kPhaseAll);

}  // namespace cg
