// Fixed device scratch for callers that cannot allocate device memory
// (pcr_retrieve_static in include/pcr.h).
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it until the process exits.  Its name is only a host-side
// handle: host code must not hand `g_scratch` itself to a kernel.  The device
// address is looked up once per device, with that device current, through
// cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pcr_internal.h"

namespace pcr {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

void* static_scratch(size_t* cap, std::string* why) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *why = "device index out of range";
    return nullptr;
  }
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      *why = cudaGetErrorString(e);
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  *cap = kStaticScratchBytes;
  return g_scratch_addr[dev];
}

}  // namespace pcr
