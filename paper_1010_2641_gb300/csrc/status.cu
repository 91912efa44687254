// Status codes, per-thread error messages and logging switch of libscatter.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include "scatter_internal.h"

namespace scatter {

namespace {
thread_local char g_last_error[512] = "";
}

scatter_status fail(scatter_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  if (log_enabled()) fprintf(stderr, "[scatter] %s: %s\n", scatter_status_string(st), g_last_error);
  return st;
}

scatter_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SCATTER_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(SCATTER_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) {
    cudaGetLastError();
    return fail(SCATTER_ERR_NO_DEVICE, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(SCATTER_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool log_enabled() {
  static int flag = -1;
  if (flag < 0) {
    const char* v = getenv("SCATTER_LOG");
    flag = (v && v[0] == '1') ? 1 : 0;
  }
  return flag == 1;
}

bool injected_alloc_failure() {
  static std::mutex mu;
  static std::string seen;
  static long count = 0;
  const char* v = getenv("SCATTER_FAULT");
  std::lock_guard<std::mutex> lock(mu);
  if (!v || strncmp(v, "alloc", 5) != 0) {
    seen.clear();
    count = 0;
    return false;
  }
  if (seen != v) {
    seen = v;
    count = 0;
  }
  const long n = v[5] == ':' ? atol(v + 6) : 1;
  return ++count == n;
}

}  // namespace scatter

extern "C" const char* scatter_status_string(scatter_status s) {
  switch (s) {
    case SCATTER_OK: return "SCATTER_OK";
    case SCATTER_ERR_INVALID_ARG: return "SCATTER_ERR_INVALID_ARG";
    case SCATTER_ERR_UNSUPPORTED: return "SCATTER_ERR_UNSUPPORTED";
    case SCATTER_ERR_OOM: return "SCATTER_ERR_OOM";
    case SCATTER_ERR_CUDA: return "SCATTER_ERR_CUDA";
    case SCATTER_ERR_TIMEOUT: return "SCATTER_ERR_TIMEOUT";
    case SCATTER_ERR_NUMERIC: return "SCATTER_ERR_NUMERIC";
    case SCATTER_ERR_NO_DEVICE: return "SCATTER_ERR_NO_DEVICE";
  }
  return "SCATTER_ERR_UNKNOWN";
}

extern "C" const char* scatter_last_error(void) { return scatter::g_last_error; }
