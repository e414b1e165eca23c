// ff.cuh -- float-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2
// (about 48 significant bits), built from the error-free transformations
// TwoSum (Knuth) and TwoProduct by FMA (Dekker's product with a fused
// multiply-add).  The _rn intrinsics keep the compiler from contracting a
// product into the following sum, which would break the error terms.
#pragma once
#include <cuda_runtime.h>

// hi + lo from s + e, |s| >= |e| or s + e exact (Fast2Sum)
__device__ __forceinline__ float2 ff_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

struct NumFF {
  using T = float2;  // (hi, lo)
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  // a b: TwoProduct of the high parts plus the cross terms (the lo * lo term is
  // below the format's precision), renormalised
  static __device__ __forceinline__ T mul(T a, T b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return ff_fast(p, e);
  }
  // a b + c: TwoProduct of the high parts, TwoSum with c's high part, the
  // cross terms and both low parts collected, renormalised
  static __device__ __forceinline__ T fma(T a, T b, T c) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    const float s = __fadd_rn(p, c.x);
    const float v = __fsub_rn(s, p);
    const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(c.x, v));
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    e = __fadd_rn(e, __fadd_rn(c.y, err));
    return ff_fast(s, e);
  }
  static __device__ __forceinline__ T fms(T a, T b, T c) { return fma(make_float2(-a.x, -a.y), b, c); }
  // v (-1)^k: sign bits flipped on the integer pipe
  static __device__ __forceinline__ T flip(T v, int k) {
    const unsigned m = (unsigned)(k & 1) << 31;
    return make_float2(__uint_as_float(__float_as_uint(v.x) ^ m), __uint_as_float(__float_as_uint(v.y) ^ m));
  }
  static __device__ __forceinline__ float f32(T v) { return v.x; }  // hi = RN(hi + lo)
};
