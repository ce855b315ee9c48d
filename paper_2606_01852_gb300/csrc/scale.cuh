// Exponent scaling (device side): the exact powers of two by which a tensor is
// renormalised, and the binary exponent of a stored value.
#pragma once

#include <cstdint>

#include "kernels.h"

namespace tn {

// floor(log2 |v|) from the IEEE-754 exponent field; very small values map to -127.
__device__ __forceinline__ int exp_of(float v) {
  return ((__float_as_int(v) >> 23) & 0xff) - 127;
}

// 2^-e as a float, e clamped to the normal range.
__device__ __forceinline__ float pow2_neg(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((127 - e) << 23);
}

// The exponent a consumer divides a tensor by (its largest stored exponent); an all-zero
// tensor is not rescaled.
__device__ __forceinline__ int scale_exp(const ScaleRec* r) {
  int e = r->emax;
  return e < -126 ? 0 : e;
}

}  // namespace tn
