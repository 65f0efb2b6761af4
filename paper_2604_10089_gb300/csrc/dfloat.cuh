// Double-FP32 ("double-float") arithmetic shared by the refinement-residual
// pair sums.
#pragma once
#include <cuda_runtime.h>

// Every quantity is an unevaluated sum hi + lo of two floats; sums and
// products use the error-free transformations TwoSum (Knuth) and TwoProd (one
// FMA), renormalised with Fast2Sum (Dekker).  Relative accuracy per operation
// is about 2^-44, so (K phi)_p is accurate to ~1e-13 of its terms while
// running on the FP32 pipe (64x the FP64 rate on GB300).  The reciprocal
// square root is a MUFU seed refined by one Newton step in double-float.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl df_split(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

// Packed double-float arithmetic on two lanes at once (FP32x2 instructions):
// every D2 holds two independent double-float numbers (the terms of two source
// nodes for one target, or of two targets for one source).  Intermediate results stay
// unnormalised (lo may exceed half an ulp of hi by a few ulps; the dropped
// lo*lo products are then ~2^-44 of the operands' product) and are
// renormalised with Fast2Sum only where cancellation is expected (the
// separation r and the dot products r.n, r.(phi_q - phi_p)), after the
// Newton step of |r|^-1, and in the running sums.
struct D2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b, rounded once
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// TwoSum (Knuth): s + e = a + b exactly.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ D2 fast2sum2(float2 a, float2 b) {   // |a| >= |b|
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ D2 dadd_u(D2 a, D2 b) {
  float2 s, e;
  two_sum2(a.hi, b.hi, s, e);
  return {s, add2(e, add2(a.lo, b.lo))};
}
__device__ __forceinline__ D2 dadd_n(D2 a, D2 b) {
  const D2 t = dadd_u(a, b);
  return fast2sum2(t.hi, t.lo);
}
// TwoProd by FMA plus the cross terms.
__device__ __forceinline__ D2 dmul_u(D2 a, D2 b) {
  const float2 p = mul2(a.hi, b.hi);
  float2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  return {p, e};
}
__device__ __forceinline__ D2 dsq_u(D2 a) {
  const float2 p = mul2(a.hi, a.hi);
  float2 e = fma2(a.hi, a.hi, neg2(p));
  e = fma2(a.hi, add2(a.lo, a.lo), e);
  return {p, e};
}


// Scalar double-float sum, renormalised (TwoSum, then Fast2Sum): the packed
// sum above on duplicated lanes, so every double-float addition of the pair
// sums goes through the same FP32x2 instruction sequence.
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const D2 r = dadd_n({f2(a.hi), f2(a.lo)}, {f2(b.hi), f2(b.lo)});
  return {r.hi.x, r.lo.x};
}
