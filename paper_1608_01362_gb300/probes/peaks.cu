// Roofline denominators for the row gathers, measured on the GPU at hand:
// the rate at which a GPU-filling grid reads rows chosen at random from a
// table (L2-resident or not), and the rate of random 4-byte lookups in each
// SM's shared memory.  The gathers of the method (Algorithm 3's reads of a
// source's contribution, a CF factor row, a PPR vector row) are bound by one
// of these rather than by a streaming HBM copy.
#include <algorithm>

#include "common.cuh"

namespace cg {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kRowsInFlight = 4;

// Rows of ROW bytes: ROW/32 lanes read 32 bytes each (two 16-byte loads);
// 4-byte rows: one lane reads one value.  Row indices come from a per-group
// LCG, masked to the table's power-of-two row count.
template <int ROW>
__global__ void __launch_bounds__(kProbeThreads, 2)
row_probe_kernel(const uint4* __restrict__ table, uint32_t row_mask, int iters,
                 float* __restrict__ sink) {
  constexpr int L = ROW >= 32 ? ROW / 32 : 1;
  const int lane = threadIdx.x & 31, sub = lane % L;
  uint32_t h = ((blockIdx.x * (uint32_t)kProbeThreads + threadIdx.x) / L) * 2654435761u + 777u;
  float acc = 0.0f;
  for (int i = 0; i < iters; ++i) {
    uint4 v[kRowsInFlight], w[kRowsInFlight];
#pragma unroll
    for (int u = 0; u < kRowsInFlight; ++u) {
      h = h * 1664525u + 1013904223u;
      const uint32_t r = (h >> 6) & row_mask;
      if (ROW >= 32) {
        const uint4* p = table + (size_t)r * (ROW / 16) + sub * 2;
        v[u] = __ldg(p);
        w[u] = __ldg(p + 1);
      } else {
        const float x = __ldg(reinterpret_cast<const float*>(table) + r);
        v[u] = make_uint4(__float_as_uint(x), 0u, 0u, 0u);
        w[u] = v[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kRowsInFlight; ++u)
      acc += __uint_as_float(v[u].x ^ w[u].y) + __uint_as_float(v[u].z ^ w[u].w);
  }
  if (acc == 1234.5f) sink[0] = acc;  // keeps the loads; never true for a zero table
}

constexpr int kSmemTable = 32768;  // 128 KB of 4-byte entries

__global__ void __launch_bounds__(kProbeThreads, 1)
smem_probe_kernel(int iters, float* __restrict__ sink) {
  extern __shared__ float tab[];
  for (int i = threadIdx.x; i < kSmemTable; i += kProbeThreads) tab[i] = (float)i;
  __syncthreads();
  uint32_t h = (blockIdx.x * (uint32_t)kProbeThreads + threadIdx.x) * 2654435761u + 12345u;
  float acc = 0.0f;
  for (int i = 0; i < iters; ++i) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      h = h * 1664525u + 1013904223u;
      v[u] = tab[(h >> 9) & (kSmemTable - 1)];
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) acc += v[u];
  }
  if (acc == 1234.5f) sink[0] = acc;
}

// Average seconds of `reps` launches after one warm-up launch.
template <class Launch>
int time_launches(Launch launch, int reps, cudaStream_t s, double* seconds) {
  cudaEvent_t a = nullptr, b = nullptr;
  CG_CUDA(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "probe launch", __FILE__, __LINE__);
  *seconds = ms / 1e3 / reps;
  return CG_OK;
}

template <int ROW>
int row_probe(const uint4* table, int64_t table_bytes, int sm_count, float* sink, cudaStream_t s,
              double* bytes_per_s) {
  const int64_t rows = table_bytes / ROW;
  uint32_t mask = 1;  // largest power of two <= rows, minus one
  while ((int64_t)(mask + 1) * 2 <= rows && mask < 0x7FFFFFFFu) mask = mask * 2 + 1;
  constexpr int L = ROW >= 32 ? ROW / 32 : 1;
  const int grid = 2 * sm_count;
  const int64_t groups = (int64_t)grid * kProbeThreads / L;
  // about 8 GB (rows) or 1 G reads (4-byte values) per launch
  const double per_launch = ROW >= 32 ? 8e9 / ROW : 1e9;
  const int iters = (int)std::max<int64_t>(1, (int64_t)(per_launch / (groups * kRowsInFlight)));
  double sec = 0.0;
  CG_TRY(time_launches(
      [&] { row_probe_kernel<ROW><<<grid, kProbeThreads, 0, s>>>(table, mask, iters, sink); }, 3,
      s, &sec));
  *bytes_per_s = (double)groups * kRowsInFlight * iters * ROW / sec;
  return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" int cg_measure_row_gather(int32_t row_bytes, int64_t table_bytes,
                                     double* bytes_per_s, cudaStream_t stream) {
  CG_ARG(bytes_per_s != nullptr, "cg_measure_row_gather: null output");
  CG_ARG(row_bytes == 4 || row_bytes == 128 || row_bytes == 256,
         "cg_measure_row_gather: row_bytes must be 4, 128 or 256 (got %d)", row_bytes);
  CG_ARG(table_bytes >= (int64_t)2 * row_bytes && table_bytes <= ((int64_t)8 << 30),
         "cg_measure_row_gather: table_bytes must be in [2 rows, 8 GiB] (got %lld)",
         (long long)table_bytes);
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  uint4* table = nullptr;
  float* sink = nullptr;
  CG_CUDA(cudaMalloc((void**)&table, (size_t)table_bytes));
  cudaError_t e = cudaMalloc((void**)&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(table, 0, (size_t)table_bytes, stream);
  int rc = CG_OK;
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "cg_measure_row_gather: table", __FILE__, __LINE__);
  } else if (row_bytes == 4) {
    rc = row_probe<4>(table, table_bytes, di.sm_count, sink, stream, bytes_per_s);
  } else if (row_bytes == 128) {
    rc = row_probe<128>(table, table_bytes, di.sm_count, sink, stream, bytes_per_s);
  } else {
    rc = row_probe<256>(table, table_bytes, di.sm_count, sink, stream, bytes_per_s);
  }
  cudaStreamSynchronize(stream);
  cudaFree(sink);
  cudaFree(table);
  return rc;
}

extern "C" int cg_measure_smem_lookups(double* lookups_per_s, cudaStream_t stream) {
  CG_ARG(lookups_per_s != nullptr, "cg_measure_smem_lookups: null output");
  DeviceInfo di{};
  CG_TRY(device_info(&di));
  float* sink = nullptr;
  CG_CUDA(cudaMalloc((void**)&sink, sizeof(float)));
  const size_t smem = kSmemTable * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute((const void*)smem_probe_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int rc = CG_OK;
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "cg_measure_smem_lookups: shared memory", __FILE__, __LINE__);
  } else {
    const int grid = di.sm_count, iters = 2048;  // 16 lookups per thread per iteration
    double sec = 0.0;
    rc = time_launches(
        [&] { smem_probe_kernel<<<grid, kProbeThreads, smem, stream>>>(iters, sink); }, 3, stream,
        &sec);
    if (rc == CG_OK) *lookups_per_s = (double)grid * kProbeThreads * 16.0 * iters / sec;
  }
  cudaFree(sink);
  return rc;
}
