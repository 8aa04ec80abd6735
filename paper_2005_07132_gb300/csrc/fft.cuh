// Shared-memory Stockham FFT building blocks (radix 8 with a final radix 4
// or 2 pass) for power-of-two lengths, used by the discrete Hilbert transform
// of the per-spectrum KK path and of the basis vectors.
//
// Stockham autosort pass with radix R over a length-L sequence whose current
// sub-transforms have length Ns: butterfly j (0 <= j < L/R) reads the R
// inputs x[j + r L/R], twiddles input r by w_{Ns R}^{(j mod Ns) r}, takes an
// R-point DFT and writes output s to y[(j div Ns) Ns R + (j mod Ns) + s Ns].
// After all passes (Ns = 1, R1, R1 R2, ...) y holds the DFT in natural order.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"

namespace fkk {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiply by SIGN*i
template <int SIGN>
__device__ __forceinline__ float2 c_rot(float2 a) {
  return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = c_add(a, b);
  v[1] = c_sub(a, b);
}

// X_s = sum_r v_r w^{rs}, w = exp(SIGN 2 pi i / 4) = SIGN*i
template <int SIGN>
__device__ __forceinline__ void dft4(float2* v) {
  float2 s02 = c_add(v[0], v[2]), d02 = c_sub(v[0], v[2]);
  float2 s13 = c_add(v[1], v[3]), d13 = c_rot<SIGN>(c_sub(v[1], v[3]));
  v[0] = c_add(s02, s13);
  v[2] = c_sub(s02, s13);
  v[1] = c_add(d02, d13);
  v[3] = c_sub(d02, d13);
}

// radix 8 as two radix-4 DFTs (even / odd inputs) and a twiddled combine
template <int SIGN>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<SIGN>(e);
  dft4<SIGN>(o);
  const float c = 0.70710678118654752f;
  // w8^s o_s for s = 0..3, w8 = c (1 + SIGN i)
  float2 t1 = make_float2(c * (o[1].x - SIGN * o[1].y), c * (o[1].y + SIGN * o[1].x));
  float2 t2 = c_rot<SIGN>(o[2]);
  float2 t3 = make_float2(c * (-o[3].x - SIGN * o[3].y), c * (-o[3].y + SIGN * o[3].x));
  v[0] = c_add(e[0], o[0]);
  v[4] = c_sub(e[0], o[0]);
  v[1] = c_add(e[1], t1);
  v[5] = c_sub(e[1], t1);
  v[2] = c_add(e[2], t2);
  v[6] = c_sub(e[2], t2);
  v[3] = c_add(e[3], t3);
  v[7] = c_sub(e[3], t3);
}

template <int R, int SIGN>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 8) dft8<SIGN>(v);
  else if constexpr (R == 4) dft4<SIGN>(v);
  else dft2<SIGN>(v);
}

// One Stockham pass.  tw[t] = exp(-2 pi i t / L) (forward table); SIGN=+1
// uses its conjugate.  Threads t0, t0+nt, ... of the calling group share the
// L/R butterflies.
template <int R, int SIGN>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ x, float2* __restrict__ y,
                                              int L, int Ns, const float2* __restrict__ tw, int t0,
                                              int nt) {
  const int LR = L / R;
  const int tws = L / (Ns * R);
  for (int j = t0; j < LR; j += nt) {
    const int k = j & (Ns - 1);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 a = x[j + r * LR];
      if (r > 0 && Ns > 1) {
        float2 w = tw[k * r * tws];
        if (SIGN > 0) w.y = -w.y;
        a = c_mul(a, w);
      }
      v[r] = a;
    }
    dftR<R, SIGN>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[base + r * Ns] = v[r];
  }
}

// Full length-L transform (L a power of two, 2 <= L).  Input in buf[0];
// returns the buffer index (0 or 1) holding the result.  Every pass ends with
// a __syncthreads(), so all threads of the block must call it together.
template <int SIGN>
__device__ __forceinline__ int fft_block(float2* buf0, float2* buf1, int L, const float2* tw, int t0,
                                         int nt) {
  float2* bufs[2] = {buf0, buf1};
  int cur = 0;
  int Ns = 1;
  while (Ns < L) {
    int rem = L / Ns;
    if (rem >= 8) {
      stockham_pass<8, SIGN>(bufs[cur], bufs[cur ^ 1], L, Ns, tw, t0, nt);
      Ns *= 8;
    } else if (rem == 4) {
      stockham_pass<4, SIGN>(bufs[cur], bufs[cur ^ 1], L, Ns, tw, t0, nt);
      Ns *= 4;
    } else {
      stockham_pass<2, SIGN>(bufs[cur], bufs[cur ^ 1], L, Ns, tw, t0, nt);
      Ns *= 2;
    }
    cur ^= 1;
    __syncthreads();
  }
  return cur;
}

// Fill tw[t] = exp(-2 pi i t / L), t < L (block-cooperative; caller syncs).
__device__ __forceinline__ void fill_twiddles(float2* tw, int L) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)L, &s, &c);
    tw[t] = make_float2(c, s);
  }
}

// Multiply bin m of a length-L spectrum by -i*sgn(m) (0 at DC and Nyquist):
// the Fourier multiplier of the discrete Hilbert transform.
__device__ __forceinline__ float2 hilbert_mult(float2 z, int m, int L) {
  if (m == 0 || 2 * m == L) return make_float2(0.f, 0.f);
  return (2 * m < L) ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
}

// ------------------------------------------------------- double-word ---
// Double-word complex variants for the k basis vectors (a few rows of length
// L): a complex number is a dw2 pair, lane x the real part and lane y the
// imaginary part (about 48 bits each), on the fp32 pipe -- this part's fp64
// rate would make an fp64 transform of the rows several times slower.
using dz = dw2::df2;

__device__ __forceinline__ dz dz_mul(dz a, dz b) {
  // (re a re b - im a im b, re a im b + im a re b)
  const dz ar = {make_float2(a.h.x, a.h.x), make_float2(a.l.x, a.l.x)};
  const dz ai = {make_float2(a.h.y, a.h.y), make_float2(a.l.y, a.l.y)};
  const dz bs = {make_float2(-b.h.y, b.h.x), make_float2(-b.l.y, b.l.x)};
  return dw2::add(dw2::mul(ar, b), dw2::mul(ai, bs));
}

// One radix-2 Stockham pass (same indexing as above).
template <int SIGN>
__device__ __forceinline__ void stockham_pass2_dz(const dz* __restrict__ x, dz* __restrict__ y, int L, int Ns,
                                                  const dz* __restrict__ tw, int t0, int nt) {
  const int LR = L / 2;
  const int tws = L / (Ns * 2);
  for (int j = t0; j < LR; j += nt) {
    const int k = j & (Ns - 1);
    const dz a = x[j];
    dz b = x[j + LR];
    if (Ns > 1) {
      dz w = tw[k * tws];
      if (SIGN > 0) {
        w.h.y = -w.h.y;
        w.l.y = -w.l.y;
      }
      b = dz_mul(b, w);
    }
    const int base = (j - k) * 2 + k;
    y[base] = dw2::add(a, b);
    y[base + Ns] = dw2::sub(a, b);
  }
}

template <int SIGN>
__device__ __forceinline__ int fft_block_dz(dz* buf0, dz* buf1, int L, const dz* tw, int t0, int nt) {
  dz* bufs[2] = {buf0, buf1};
  int cur = 0;
  for (int Ns = 1; Ns < L; Ns *= 2) {
    stockham_pass2_dz<SIGN>(bufs[cur], bufs[cur ^ 1], L, Ns, tw, t0, nt);
    cur ^= 1;
    __syncthreads();
  }
  return cur;
}

// Multiply by -i*sgn(m) (0 at DC and Nyquist), exactly.
__device__ __forceinline__ dz hilbert_mult_dz(dz z, int m, int L) {
  if (m == 0 || 2 * m == L) return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  if (2 * m < L) return {make_float2(z.h.y, -z.h.x), make_float2(z.l.y, -z.l.x)};
  return {make_float2(-z.h.y, z.h.x), make_float2(-z.l.y, z.l.x)};
}

}  // namespace fkk
