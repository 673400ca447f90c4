// Allocation-free gradient J^T r (gn_jtr_noalloc).
//
// Every other entry point works through a handle whose workspace gn_init
// allocates with cudaMalloc.  Some callers cannot do that: code running
// inside a host application that owns all device memory through its own
// allocator (a raw cudaMalloc there can fail or fragment the pool), loops
// that must not pay the device-wide synchronisation that cudaMalloc/cudaFree
// may imply, and plug-ins that only ever receive device pointers from their
// host.  For them this file offers J^T r on caller-owned buffers with its
// scratch in a fixed, file-scope device array instead of allocated memory.
//
// The scratch (kGemvChunks x 16384 doubles = 8 MiB) is part of the module
// image: every GPU that loads libgn holds it until the process exits.  Its
// device address is looked up once per device (cudaGetSymbolAddress, with
// that device current) on the first call made on that device; make that
// first call before any stream capture.  All calls on a device share the
// array and it keeps the contents of the last call; no clearing is needed
// because every scratch entry a call reads is written earlier by the same
// call.  Calls whose executions overlap on the GPU (different streams, or
// different host threads on one device) race on the scratch: serialise them.
// The looked-up address stays cached for the life of the process; it is not valid
// across a cudaDeviceReset of that device (the module is then loaded anew), so callers
// that reset a device must not call this entry point on it afterwards.
#include <mutex>

#include "gn_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxCols = 16384;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[gn::kGemvChunks * kNoAllocMaxCols];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocMaxDevices];

}  // namespace

extern "C" int gn_jtr_noalloc(const double* J, int64_t ld, int64_t nrows, int64_t ncols, const double* r,
                              double* g_out, void* cuda_stream) {
  if (!J || !r || !g_out || nrows < 0 || ncols < 1 || ld < ncols) return GN_ERR_INVALID;
  if (ncols > kNoAllocMaxCols) return GN_ERR_TOO_LARGE;
  int dev = -1;
  if (GN_NOTE(cudaGetDevice(&dev)) != cudaSuccess) return GN_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GN_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (GN_NOTE(cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess || !p) return GN_ERR_CUDA;
      g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_addr[dev];
  }
  const cudaError_t e = GN_NOTE(
      gn::dgemv_t_scratch(J, ld, nrows, ncols, r, g_out, 0.0, scratch, static_cast<cudaStream_t>(cuda_stream)));
  return e == cudaSuccess ? GN_OK : GN_ERR_CUDA;
}
