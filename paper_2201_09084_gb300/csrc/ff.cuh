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


// One split-part pair advance with float-float storage: each part
// F <- ea F + eb (r + source); returns the rounded total of both parts.
__device__ __forceinline__ float advff(float2* p0, float2* p1, long long id, float r0, float r1, float src, float2 ea0,
                                       float2 eb0, float2 ea1, float2 eb1, bool into1) {
  const float2 a = p0[id], b = p1[id];
  ff e0 = ff_add(ff_mul(ea0, ff{a.x, a.y}), ff_mul(eb0, ff_two_sum(r0, into1 ? 0.f : src)));
  ff e1 = ff_add(ff_mul(ea1, ff{b.x, b.y}), ff_mul(eb1, ff_two_sum(r1, into1 ? src : 0.f)));
  p0[id] = make_float2(e0.h, e0.l);
  p1[id] = make_float2(e1.h, e1.l);
  const ff t = ff_add(e0, e1);
  return __fadd_rn(t.h, t.l);
}

}  // namespace picpml
