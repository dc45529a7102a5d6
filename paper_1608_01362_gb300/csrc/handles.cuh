// Library-owned handle layouts (opaque to C callers).
#pragma once

#include <vector>

#include "seg_gather.cuh"

// The segmented graph of Algorithm 2, flattened: all subgraphs concatenated
// in segment order.  Subgraph row i (global row index over all segments)
// holds edges [row_ptr[i], row_ptr[i+1]) (stored flagged and padded in
// plan.colf) and its destination is idx_map[i].  blk[b*k + s] is the first
// (global) row of segment s whose destination is >= b*B (block-major: a
// merge block's starts of all segments are contiguous); rows of segment s
// inside merge block b are [blk[b*k + s], blk[(b+1)*k + s]).
struct cg_segmented {
  int device = 0;
  int32_t V = 0;
  int64_t E = 0;
  int32_t k = 0;
  int32_t B = 0;
  int32_t nb = 0;
  int64_t rows = 0;
  std::vector<int64_t> bounds, row_base, edge_base;  // host copies, k+1 each
  int32_t* row_ptr = nullptr;  // [rows+1] (export only; the gather reads flagged edges)
  int32_t* idx_map = nullptr;  // [rows]
  int32_t* blk = nullptr;      // [(nb+1)*k] block-major
  cg::SegPlan plan;            // flagged padded edges + chunk index + launch shape
  void* interm = nullptr;        // [rows] 4-byte values (intermBuf)
  double* partials = nullptr;    // [2*nb] per-block FP64 partial sums
  unsigned* counter = nullptr;   // last-block detection
  double* dslot = nullptr;       // [4] FP64 iteration state (dangling ping-pong, scratch)
  float* rank_tmp = nullptr;     // [V] ping-pong for multi-iteration calls
  float* contrib_tmp = nullptr;  // [V]
  int64_t bytes = 0;
};

// The plain pull baseline: the caller's CSR plus a merge-path tiling.
struct cg_plain {
  int device = 0;
  int32_t V = 0;
  int64_t E = 0;
  const int64_t* offsets = nullptr;  // caller-owned
  const int32_t* src = nullptr;      // caller-owned
  cg::TilePlan plan;
  float* acc = nullptr;          // [V] gathered sums
  double* partials = nullptr;    // [2*nb]
  unsigned* counter = nullptr;
  double* dslot = nullptr;       // [4]
  float* rank_tmp = nullptr;
  float* contrib_tmp = nullptr;
  int32_t nb = 0;
  int64_t bytes = 0;
};

namespace cg {
// Validate an in-edge CSR on the device (offsets monotone from 0 to E, every
// source in [0, V)).  Synchronizes the stream.
int validate_csr(const int64_t* offsets, const int32_t* src, int32_t V, int64_t E,
                 cudaStream_t s);
}  // namespace cg
