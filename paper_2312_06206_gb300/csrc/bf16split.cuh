// bf16split.cuh -- FP32 value -> BF16 pair (hi, lo) with v ~= hi + lo:
// hi = v rounded to the nearest BF16, lo = (v - hi) rounded to the nearest
// BF16 (v - hi is exact in FP32).  |v - hi - lo| <= 2^-16 |v|.
#pragma once
#include <cuda_bf16.h>

namespace sadi {

__device__ __forceinline__ void split_bf16(float v, unsigned short* hi, unsigned short* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *hi = __bfloat16_as_ushort(h);
  *lo = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
}

}  // namespace sadi
