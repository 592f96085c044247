// Library-owned scratch for atlas_nabla_laplacian_edges_noalloc.
//
// Some callers cannot call cudaMalloc at the point where they apply the
// operator: code that runs inside another framework's memory pool or a
// pre-sized arena (every byte of device memory handed out up front), code
// running between phases that must not allocate or synchronise, and callers
// that have no allocator of their own (a Fortran model calling through the
// C ABI with only field pointers).  The two-pass Laplacian needs scratch for
// its edge fluxes and the intermediate gradient; this file provides it as a
// file-scope device array, so that the entry point allocates nothing.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (kScratchBytes) until the process exits.  Its device
// address is looked up once per device (cudaGetSymbolAddress) on the first
// call made with that device current; that first call should therefore come
// before any stream capture.  The address stays cached: after a
// cudaDeviceReset, which also invalidates every fvm's device tables, the
// entry point must not be called again in the process.  All calls on a
// device share the array and it keeps the last call's contents; calls that
// overlap on the GPU (different streams without ordering) race on it.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "kernels.h"

namespace atlasgb {

namespace {
constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
}  // namespace

size_t noalloc_scratch_bytes() { return kScratchBytes; }

// Device address of the scratch array on the current device (looked up once
// per device).  Returns cudaSuccess and the pointer, or the CUDA error.
cudaError_t noalloc_scratch(void** ptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *ptr = g_addr[dev];
  return cudaSuccess;
}

}  // namespace atlasgb
