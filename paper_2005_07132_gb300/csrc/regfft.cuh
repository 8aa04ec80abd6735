// In-register radix-2 FFTs of compile-time length for one thread's values,
// with the butterfly twiddles folded to compile-time constants.
//
// fft_dif<N, SIGN>: natural-order input, bit-reversed output
//   (x[i] <- X[bitrev_N(i)]),
// fft_dit<N, SIGN>: bit-reversed input, natural-order output,
// both computing X[k] = sum_n x[n] exp(SIGN 2 pi i n k / N), unnormalised
// (SIGN = -1 forward, +1 inverse).  Every index is a template constant, so
// the register array is never addressed dynamically; multiplications by 1,
// +-i and (+-1 +-i)/sqrt(2) are specialised.  The twiddle constants are
// evaluated by the host compiler from a Taylor series (cx_cos / cx_sin
// below) and rounded to float.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace fkk {
namespace rf {

template <int I, int N, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }
constexpr int bitrev(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}

// sin / cos of 2 pi e / n, argument reduced to [-pi, pi], 30 Taylor terms
// in double (error far below float rounding).
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double cx_angle(int e, int n) {
  const int r = ((e % n) + n) % n;
  return kTwoPi * (double)(2 * r <= n ? r : r - n) / (double)n;
}
constexpr double cx_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 30; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double cx_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 30; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}

// Complex add / subtract: one paired fp32 instruction (FADD2) on the device.
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}

// v * exp(SIGN 2 pi i E / N)
template <int SIGN, int E, int N>
__host__ __device__ __forceinline__ float2 twiddle(float2 v) {
  constexpr int e = ((E % N) + N) % N;
  if constexpr (e == 0) {
    return v;
  } else if constexpr (4 * e == N) {  // SIGN * i
    return SIGN < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  } else if constexpr (2 * e == N) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * e == 3 * N) {  // -SIGN * i
    return SIGN < 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else if constexpr (8 * e == N || 8 * e == 3 * N || 8 * e == 5 * N || 8 * e == 7 * N) {
    constexpr float h = 0.70710678118654752440f;
    constexpr float cr = (8 * e == N || 8 * e == 7 * N) ? h : -h;
    constexpr float sr = (8 * e == N || 8 * e == 3 * N) ? h : -h;  // sin of the angle
    constexpr float ci = SIGN * sr;
    // (v.x + i v.y)(cr + i ci)
    return make_float2(cr * v.x - ci * v.y, cr * v.y + ci * v.x);
  } else {
    constexpr float c = (float)cx_cos(cx_angle(e, N));
    constexpr float s = (float)(SIGN * cx_sin(cx_angle(e, N)));
    return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
  }
}

template <int N, int SIGN, int OFF = 0>
__host__ __device__ __forceinline__ void fft_dif(float2* x) {
  constexpr int S = ilog2(N);
  static_for<0, S>([&](auto st) {
    constexpr int span = N >> (decltype(st)::value + 1);
    static_for<0, N / 2>([&](auto b) {
      constexpr int bi = decltype(b)::value;
      constexpr int g = (bi / span) * 2 * span, j = bi % span;
      const float2 a = x[OFF + g + j], c = x[OFF + g + j + span];
      x[OFF + g + j] = cadd(a, c);
      x[OFF + g + j + span] = twiddle<SIGN, j * (N / (2 * span)), N>(csub(a, c));
    });
  });
}

template <int N, int SIGN, int OFF = 0>
__host__ __device__ __forceinline__ void fft_dit(float2* x) {
  constexpr int S = ilog2(N);
  static_for<0, S>([&](auto st) {
    constexpr int span = 1 << decltype(st)::value;
    static_for<0, N / 2>([&](auto b) {
      constexpr int bi = decltype(b)::value;
      constexpr int g = (bi / span) * 2 * span, j = bi % span;
      const float2 a = x[OFF + g + j];
      const float2 c = twiddle<SIGN, j * (N / (2 * span)), N>(x[OFF + g + j + span]);
      x[OFF + g + j] = cadd(a, c);
      x[OFF + g + j + span] = csub(a, c);
    });
  });
}

}  // namespace rf
}  // namespace fkk
