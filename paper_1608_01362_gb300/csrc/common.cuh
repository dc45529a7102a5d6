// Shared host/device helpers of the cagra_gb CUDA library: status codes,
// thread-local error text, device properties, block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/cagra_gb.h"

namespace cg {

// Thread-local last error text (read through cg_last_error_message()).
void set_error(const char* fmt, ...);
const char* last_error();

// Record a CUDA error and return CG_ERR_CUDA (or CG_ERR_OOM).
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CG_CUDA(call)                                                      \
  do {                                                                     \
    cudaError_t cg_e_ = (call);                                            \
    if (cg_e_ != cudaSuccess)                                              \
      return ::cg::cuda_fail(cg_e_, #call, __FILE__, __LINE__);            \
  } while (0)

#define CG_LAUNCH_CHECK()                                                  \
  do {                                                                     \
    cudaError_t cg_e_ = cudaGetLastError();                                \
    if (cg_e_ != cudaSuccess)                                              \
      return ::cg::cuda_fail(cg_e_, "kernel launch", __FILE__, __LINE__);  \
  } while (0)

#define CG_ARG(cond, ...)                                                  \
  do {                                                                     \
    if (!(cond)) {                                                         \
      ::cg::set_error(__VA_ARGS__);                                        \
      return CG_ERR_INVALID_ARG;                                           \
    }                                                                      \
  } while (0)

#define CG_TRY(expr)                                                       \
  do {                                                                     \
    int cg_s_ = (expr);                                                    \
    if (cg_s_ != CG_OK) return cg_s_;                                      \
  } while (0)

struct DeviceInfo {
  int device;
  int sm_count;
  size_t l2_bytes;
  size_t smem_optin;
};
// Properties of the current device (cached per device).
int device_info(DeviceInfo* out);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Grid size for grid-stride kernels: a multiple of the SM count.
int grid_for(int64_t n, int threads, int per_sm = 8);

// ---------------------------------------------------------------------------
// Scans and sorts (scan.cu).  All stream-ordered; scratch from the stream-
// ordered allocator.
// ---------------------------------------------------------------------------
// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n+1 entries.
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
int radix_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in,
                     uint32_t* keys_out, int32_t* vals_out, int64_t n, int bits,
                     cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (result valid in thread 0).  `sh` holds >= 32 entries.
template <typename T, int THREADS>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T r = 0;
  if (w == 0) {
    r = lane < THREADS / 32 ? sh[lane] : T(0);
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// Streaming (evict-first) loads for data read once per pass.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }

}  // namespace cg
