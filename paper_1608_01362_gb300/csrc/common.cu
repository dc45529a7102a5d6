// Host-side helpers: status strings, thread-local error text, device info.
#include <stdarg.h>

#include <mutex>

#include "common.cuh"

namespace cg {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed at %s:%d: %s (%s)", what, file, line, cudaGetErrorName(e),
            cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return CG_ERR_OOM;
  }
  return CG_ERR_CUDA;
}

int device_info(DeviceInfo* out) {
  static std::mutex mu;
  static DeviceInfo cache[64];
  static bool have[64] = {false};
  int dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return CG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!have[dev]) {
    DeviceInfo d{};
    d.device = dev;
    int v = 0;
    CG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    d.sm_count = v;
    CG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev));
    d.l2_bytes = (size_t)v;
    CG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    d.smem_optin = (size_t)v;
    cache[dev] = d;
    have[dev] = true;
  }
  *out = cache[dev];
  return CG_OK;
}

int grid_for(int64_t n, int threads, int per_sm) {
  DeviceInfo di{};
  int sms = 148;
  if (device_info(&di) == CG_OK) sms = di.sm_count;
  int64_t want = ceil_div(n > 0 ? n : 1, threads);
  int64_t cap = (int64_t)sms * per_sm;
  return (int)(want < cap ? want : cap);
}

}  // namespace cg

extern "C" {

const char* cg_status_string(int status) {
  switch (status) {
    case CG_OK: return "CG_OK";
    case CG_ERR_INVALID_ARG: return "CG_ERR_INVALID_ARG";
    case CG_ERR_OOM: return "CG_ERR_OOM";
    case CG_ERR_CUDA: return "CG_ERR_CUDA";
    case CG_ERR_TIMEOUT: return "CG_ERR_TIMEOUT";
    case CG_ERR_UNSUPPORTED: return "CG_ERR_UNSUPPORTED";
    default: return "CG_ERR_UNKNOWN";
  }
}

const char* cg_last_error_message(void) { return cg::last_error(); }

int cg_version(void) { return 100; }

}  // extern "C"
