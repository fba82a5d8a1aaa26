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

namespace {
// One warp waits, as the kernels' bounded wait (mbar_wait_bounded) does but
// with `limit` tries, on an mbarrier that nothing arrives at and no copy
// completes: every lane gives up and raises GS_FLAG_TIMEOUT, as a kernel does
// when a staged copy never lands.
__global__ void wait_check_kernel(uint32_t limit, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(&bar, 0u)) return;
  atomicOr(status, GS_FLAG_TIMEOUT);
}
}  // namespace

}  // namespace gs

extern "C" gs_status gs_wait_check(uint32_t limit, int32_t* status, void* stream) {
  GS_REQUIRE(status, "gs_wait_check: null status");
  GS_REQUIRE(limit >= 1 && limit <= (1u << 20), "gs_wait_check: limit %u outside [1, 2^20]", limit);
  gs::wait_check_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(limit, status);
  return gs::check_launch("gs_wait_check");
}

extern "C" const char* gs_last_error(void) { return gs::g_err; }

extern "C" int32_t gs_version(void) { return 100; }  // 0.1.0
