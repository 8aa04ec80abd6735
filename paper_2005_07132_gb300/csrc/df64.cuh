// Double-word ("double-float") arithmetic on the fp32 pipe: a value is the
// unevaluated sum h + l of two floats with |l| <= ulp(h) / 2, about 48
// significant bits.  Built from the error-free transformations TwoSum
// (Knuth), Fast2Sum (Dekker) and the FMA-based TwoProd, with the double-word
// addition, multiplication and division algorithms analysed by Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44 (2017).
//
// The sloppy addition used throughout has an absolute error below about
// 3 u^2 (|x| + |y|) (u = 2^-24), which is what the backward-stable
// algorithms built on it need; it does not bound the relative error of a
// sum that cancels.
//
// Every rounded sum and product is written with the __fadd_rn / __fsub_rn /
// __fmul_rn intrinsics, which the compiler never contracts into an FMA: a
// contraction across these helpers would silently change a rounding the
// error-free transformations depend on.
#pragma once

#include <cuda_runtime.h>

namespace fkk {
namespace dw {

struct df {
  float h, l;
};

__device__ __forceinline__ df make(float h, float l = 0.f) { return {h, l}; }

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// |a| >= |b| (or a == 0): s + e = a + b exactly
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
// p + e = a * b exactly
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df neg(df x) { return {-x.h, -x.l}; }

// sloppy double-word addition
__device__ __forceinline__ df add(df x, df y) {
  const df s = two_sum(x.h, y.h);
  const float t = __fadd_rn(__fadd_rn(x.l, y.l), s.l);
  return fast_two_sum(s.h, t);
}
__device__ __forceinline__ df sub(df x, df y) { return add(x, neg(y)); }
__device__ __forceinline__ df add(df x, float y) {
  const df s = two_sum(x.h, y);
  return fast_two_sum(s.h, __fadd_rn(x.l, s.l));
}

// double-word times double-word (relative error about 5 u^2)
__device__ __forceinline__ df mul(df x, df y) {
  const df c = two_prod(x.h, y.h);
  const float t = fmaf(x.l, y.h, __fmul_rn(x.h, y.l));
  return fast_two_sum(c.h, __fadd_rn(c.l, t));
}
// double-word times float
__device__ __forceinline__ df mul(df x, float y) {
  const df c = two_prod(x.h, y);
  return fast_two_sum(c.h, fmaf(x.l, y, c.l));
}
// x * y + z
__device__ __forceinline__ df fma(df x, df y, df z) { return add(mul(x, y), z); }
// z - x * y
__device__ __forceinline__ df fnma(df x, df y, df z) { return sub(z, mul(x, y)); }

// double-word divided by double-word: quotient th from the leading words,
// remainder x - y th in double-word, one correction term
__device__ __forceinline__ df div(df x, df y) {
  const float th = __fdividef(x.h, y.h);
  const df r = mul(y, th);
  const float d = __fadd_rn(__fsub_rn(x.h, r.h), __fsub_rn(x.l, r.l));
  return fast_two_sum(th, __fdividef(d, y.h));
}
__device__ __forceinline__ df rcp(df y) { return div(make(1.f), y); }

// square root: s = sqrt(x.h), then one Newton correction (x - s^2) / (2 s)
__device__ __forceinline__ df sqrt(df x) {
  if (x.h <= 0.f) return make(0.f);
  const float s = sqrtf(x.h);
  const df s2 = two_prod(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, s2.h), s2.l), x.l);
  return fast_two_sum(s, __fdividef(r, __fmul_rn(2.f, s)));
}

__device__ __forceinline__ df from_double(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double to_double(df x) { return (double)x.h + (double)x.l; }

// power-of-two scaling (exact)
__device__ __forceinline__ df ldexp(df x, int e) { return {ldexpf(x.h, e), ldexpf(x.l, e)}; }

__device__ __forceinline__ bool lt0(df x) { return x.h < 0.f || (x.h == 0.f && x.l < 0.f); }
__device__ __forceinline__ float absh(df x) { return fabsf(x.h); }

__device__ __forceinline__ df shfl_xor(df x, int o) {
  return {__shfl_xor_sync(0xffffffffu, x.h, o), __shfl_xor_sync(0xffffffffu, x.l, o)};
}
__device__ __forceinline__ df shfl(df x, int src) {
  return {__shfl_sync(0xffffffffu, x.h, src), __shfl_sync(0xffffffffu, x.l, src)};
}
__device__ __forceinline__ df warp_sum(df x) {
  for (int o = 16; o > 0; o >>= 1) x = add(x, shfl_xor(x, o));
  return x;
}

}  // namespace dw

// Two independent double-word numbers carried side by side, (h.x, l.x) and
// (h.y, l.y), on Blackwell's paired fp32 instructions.  Every operation is
// dw's with the same rounding per component (the paired instructions round
// each lane as their scalar _rn forms do), so the results are bit-identical
// to two dw computations, in about half the instructions.
namespace dw2 {

struct df2 {
  float2 h, l;
};

__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 pack(dw::df a, dw::df b) { return {make_float2(a.h, b.h), make_float2(a.l, b.l)}; }
__device__ __forceinline__ df2 splat(dw::df a) { return {make_float2(a.h, a.h), make_float2(a.l, a.l)}; }

__device__ __forceinline__ df2 two_sum(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 bb = __fadd2_rn(s, neg(a));
  const float2 e = __fadd2_rn(__fadd2_rn(a, neg(__fadd2_rn(s, neg(bb)))), __fadd2_rn(b, neg(bb)));
  return {s, e};
}
__device__ __forceinline__ df2 fast_two_sum(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 e = __fadd2_rn(b, neg(__fadd2_rn(s, neg(a))));
  return {s, e};
}
__device__ __forceinline__ df2 add(df2 x, df2 y) {
  const df2 s = two_sum(x.h, y.h);
  const float2 t = __fadd2_rn(__fadd2_rn(x.l, y.l), s.l);
  return fast_two_sum(s.h, t);
}
__device__ __forceinline__ df2 sub(df2 x, df2 y) { return add(x, {neg(y.h), neg(y.l)}); }
__device__ __forceinline__ df2 mul(df2 x, df2 y) {
  const float2 p = __fmul2_rn(x.h, y.h);
  const float2 pe = __ffma2_rn(x.h, y.h, neg(p));
  const float2 t = __ffma2_rn(x.l, y.h, __fmul2_rn(x.h, y.l));
  return fast_two_sum(p, __fadd2_rn(pe, t));
}

}  // namespace dw2
}  // namespace fkk
