// gs_bin_sort_noalloc: the binning and depth sort of gs_bin_sort for callers
// that cannot allocate device memory.
//
// gs_bin_sort needs a scratch workspace (per-record tile counts and offsets, the
// second key/value buffer of the radix sort, digit histograms) that its caller
// allocates.  Some callers cannot: a process whose allocator is frozen after
// start-up (a server that reserves its HBM budget once), a plugin that only
// receives device pointers from a host framework that owns all allocation, or a
// loop that must never pay cudaMalloc's implicit device synchronisation.  This
// entry point runs the same sort with its scratch in a file-scope device array
// of fixed size that the library itself owns.
//
// The array (kScratchBytes) is part of this library's device image: every GPU
// that loads the library holds it until the process exits.  Host code cannot use
// the array's name as a device address (on the host it names a shadow object),
// so the first call on each device, with that device current, looks its device
// address up with cudaGetSymbolAddress and caches it; make that first call before
// any stream capture.  All calls share the one array and each call leaves the
// array holding its own intermediate data: calls that may overlap on the GPU
// (different streams without ordering) race on it.  Nothing in the array needs
// to start at zero: every scratch word a call reads was written earlier in the
// same call.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" gs_status gs_bin_sort_noalloc(const gs_projected* proj, int32_t n_pad, gs_frame frame, gs_sorted* out,
                                         int32_t* status, void* stream) {
  GS_REQUIRE(proj && out, "gs_bin_sort_noalloc: null argument");
  const size_t need = gs_bin_sort_workspace_size(n_pad, frame, out->capacity);
  GS_REQUIRE(need > 0, "gs_bin_sort_noalloc: bad n_pad or frame");
  GS_REQUIRE(need <= kScratchBytes,
             "gs_bin_sort_noalloc: this sort needs %zu bytes of scratch but the built-in scratch holds %zu "
             "(lower out->capacity or the views x n_pad records, or use gs_bin_sort with a workspace)",
             need, kScratchBytes);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    gs::set_error("gs_bin_sort_noalloc: no usable current device (%s)", cudaGetErrorString(e));
    return GS_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_sort_scratch);
      if (e != cudaSuccess || !p) {
        gs::set_error("gs_bin_sort_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                      cudaGetErrorString(e));
        return GS_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  return gs_bin_sort(proj, n_pad, frame, scratch, kScratchBytes, out, status, stream);
}
