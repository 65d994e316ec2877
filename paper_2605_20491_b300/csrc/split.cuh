// Split of an FP32 value into NP bf16 "planes" (x = x_0 (+ x_1 (+ x_2))): each plane is the
// round-to-nearest bf16 of what the previous planes leave; the residual subtractions are
// exact in FP32.  Planes are stored plane_stride elements apart.
#pragma once
#include <cuda_bf16.h>

namespace ts {

template <int NP>
__device__ __forceinline__ void split_store(float v, __nv_bfloat16* base, long long plane_stride, long long idx) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  base[idx] = h;
  if (NP == 1) return;
  float rres = v - __bfloat162float(h);
  __nv_bfloat16 m = __float2bfloat16_rn(rres);
  base[plane_stride + idx] = m;
  if (NP == 3) {
    float r2 = rres - __bfloat162float(m);
    base[2 * plane_stride + idx] = __float2bfloat16_rn(r2);
  }
}

}  // namespace ts
