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

// The same split of two values, returned packed (a in the low half) for one
// 4-byte store of two adjacent BF16 elements each.
__device__ __forceinline__ void split_bf16x2(float a, float b, unsigned* hi, unsigned* lo) {
  unsigned short ha, la, hb, lb;
  split_bf16(a, &ha, &la);
  split_bf16(b, &hb, &lb);
  *hi = (unsigned)ha | ((unsigned)hb << 16);
  *lo = (unsigned)la | ((unsigned)lb << 16);
}

}  // namespace sadi
