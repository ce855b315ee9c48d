// The split-BF16 storage form of a complex tensor (device side).
//
// A tensor that feeds a BF16x3 tensor-core step is written by its producer as four
// BF16 planes of E elements each, [re_hi | im_hi | re_lo | im_lo], in place of the two
// FP32 planes [re | im] (the same 8 bytes per element, so batch strides and workspace
// sizes do not change). hi = RN_bf16(v) and lo = RN_bf16(v - hi): v - hi is exact in
// FP32, so hi + lo carries 16 significant bits and |v - hi - lo| <= 2^-16 |v|.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

namespace tn {

// Store one complex value at element `off` of a tensor copy that starts at `C`
// (the copy's first float): planar FP32, or split BF16 when `split` is set.
__device__ __forceinline__ void store_cplx(float* C, int64_t plane, int64_t off, float re, float im,
                                           bool split) {
  if (!split) {
    C[off] = re;
    C[plane + off] = im;
    return;
  }
  __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(C);
  const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi = __float2bfloat16_rn(im);
  S[off] = hr;
  S[plane + off] = hi;
  S[2 * plane + off] = __float2bfloat16_rn(re - __bfloat162float(hr));
  S[3 * plane + off] = __float2bfloat16_rn(im - __bfloat162float(hi));
}

}  // namespace tn
