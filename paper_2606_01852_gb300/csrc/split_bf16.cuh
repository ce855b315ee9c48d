// The split-BF16 storage forms of a complex tensor (device side).
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

// Storage modes of a complex tensor copy (tn_storage_format): 0 planar FP32 [re | im];
// 1 split BF16 [re_hi | im_hi | re_lo | im_lo] (operands of 4M BF16x3 steps); 2 split BF16
// with the sum plane of the 3M product, [re_hi | re_lo | im_hi | im_lo | s_hi | s_lo] with
// s = re + im rounded to FP32 (operands of 3M BF16x3 steps; 12 bytes per element, each
// hi/lo pair adjacent so that one product's operand planes are one TMA box).
constexpr int kFmtPlanar = 0, kFmtSplit = 1, kFmtSplit3M = 2;

// floats per element of a complex copy in storage mode `fmt` (batch strides)
__host__ __device__ inline int64_t cplx_floats(int fmt) { return fmt == kFmtSplit3M ? 3 : 2; }

__device__ __forceinline__ void split_pair(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Store one complex value at element `off` of a tensor copy that starts at `C`
// (the copy's first float), in storage mode `fmt`.
__device__ __forceinline__ void store_cplx(float* C, int64_t plane, int64_t off, float re, float im, int fmt) {
  if (fmt == kFmtPlanar) {
    C[off] = re;
    C[plane + off] = im;
    return;
  }
  __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(C);
  __nv_bfloat16 rh, rl, ih, il;
  split_pair(re, rh, rl);
  split_pair(im, ih, il);
  if (fmt == kFmtSplit) {
    S[off] = rh;
    S[plane + off] = ih;
    S[2 * plane + off] = rl;
    S[3 * plane + off] = il;
    return;
  }
  __nv_bfloat16 sh, sl;
  split_pair(re + im, sh, sl);
  S[off] = rh;
  S[plane + off] = rl;
  S[2 * plane + off] = ih;
  S[3 * plane + off] = il;
  S[4 * plane + off] = sh;
  S[5 * plane + off] = sl;
}

}  // namespace tn
