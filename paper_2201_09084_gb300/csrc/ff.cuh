// Float-float (hi + lo) arithmetic with error-free FP32 transformations
// (Dekker, Knuth), used for the FP64-class PML split parts.
#pragma once

#include <cuda_runtime.h>

namespace picpml {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.h, b.h);
  const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return ff_quick(s.h, e);
}
__device__ __forceinline__ ff ff_mul(float2 a, ff b) {
  const float p = __fmul_rn(a.x, b.h);
  float e = __fmaf_rn(a.x, b.h, -p);
  e = __fmaf_rn(a.x, b.l, __fmaf_rn(a.y, b.h, e));
  return ff_quick(p, e);
}


}  // namespace picpml
