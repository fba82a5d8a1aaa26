// Host-side helpers of the C ABI: thread-local error text and launch checks.
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace gs {
namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

gs_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return GS_ERR_CUDA;
  }
  return GS_OK;
}

}  // namespace gs

extern "C" const char* gs_last_error(void) { return gs::g_err; }

extern "C" int32_t gs_version(void) { return 100; }  // 0.1.0
