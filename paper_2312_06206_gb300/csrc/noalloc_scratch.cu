// noalloc_scratch.cu -- the fixed device scratch area of sadi_step_noalloc.
//
// The array below is part of the library's device image: every GPU on which
// the library's device code is loaded holds its kNoallocScratchBytes until the
// process exits.  Host code never dereferences it: on the host the name only
// stands for the symbol, and its device address is looked up once per device
// with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <mutex>

#include "sadi_internal.h"

namespace sadi {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

cudaError_t noalloc_scratch_address(int device, void** out) {
  *out = nullptr;
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return e;
    if (cur != device) return cudaErrorInvalidDevice;   // the set-up needs that device current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace sadi
