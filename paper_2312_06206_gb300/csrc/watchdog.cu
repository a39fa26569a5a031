// watchdog.cu -- the state watchdog of a context: sum u_ij^2 over the grid in
// double and flag a non-finite result (a NaN or an infinity anywhere in u^n,
// or a sum that overflowed), for the failure detection of the step loop.
//
// One launch: every block reduces a grid-stride share of the state, writes
// its partial sum, and the last block to finish (ticket counter) adds the
// partials in block order -- the result does not depend on the order in
// which blocks finish -- records it with the step number, latches the
// non-finite flag (kept until the host clears it) and resets the counter for
// the next launch.
#include <cuda_runtime.h>

#include "sadi_internal.h"

namespace sadi {
namespace {

constexpr int kWdThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kWdThreads) k_watchdog(const T* __restrict__ u, size_t n, WdState* wd,
                                                         long long step) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)kWdThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kWdThreads) {
    const double v = (double)u[i];
    acc += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double warp_sum[kWdThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sum[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kWdThreads / 32; ++w) s += warp_sum[w];
    wd->partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(&wd->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double s = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) s += *(volatile double*)&wd->partial[b];
  wd->sumsq = s;
  wd->step = step;
  if (!isfinite(s) && !wd->nonfinite) {
    wd->nonfinite = 1;
    wd->nonfinite_step = step;
  }
  wd->ticket = 0;
}

}  // namespace

cudaError_t launch_watchdog(const void* u, bool fp64, size_t n, WdState* wd, long long step, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 4 * kWdThreads - 1) / (4 * kWdThreads);
  if (blocks > (size_t)kWdMaxBlocks) blocks = kWdMaxBlocks;
  if (fp64)
    k_watchdog<double><<<(unsigned)blocks, kWdThreads, 0, st>>>(static_cast<const double*>(u), n, wd, step);
  else
    k_watchdog<float><<<(unsigned)blocks, kWdThreads, 0, st>>>(static_cast<const float*>(u), n, wd, step);
  return cudaGetLastError();
}

}  // namespace sadi
