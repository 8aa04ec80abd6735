// Per-spectrum KK (Eq. KCARS with the surrogate reference of Eq. K) with the
// length-L transform held in registers: one warp per pair of spectra for
// L = 1,024, four warps per pair for L = 2,048 (kk_quad_kernel below).
//
// As in the shared-memory kernel, two real spectra share one complex FFT
// (z = a0 + i a1; the Hilbert multiplier -i sgn(m) maps it to H{a0} + i H{a1}).
// Here L = 32 R (R = 32 or 64) is split four-step style with n = n1 + 32 n2,
// k = k2 + R k1:
//   lane n1 holds z[n1 + 32 n2] for n2 = 0..R-1 -- for a fixed register the
//   32 lanes touch 32 consecutive samples, so row loads and stores coalesce;
//   1. R-point DFT over n2 in registers (compile-time twiddles),
//   2. twiddle w_L^(n1 k2) from a shared-memory table,
//   3. one transpose through a per-warp shared-memory buffer (16-byte slots,
//      XOR-swizzled, no bank conflicts) so that lane l holds all 32 n1 for
//      k2 = (R/32) l + b,
//   4. 32-point DFT over n1 in registers -> X[k2 + R k1].
// The multiplier -i sgn(k) is applied in place, and the inverse runs the same
// steps backwards (32-point DIT, conjugate twiddles, transpose, R-point DIF),
// ending with lane n1 holding sample n1 + 32 n2 again.  A warp prefetches its
// next pair of rows with cp.async into a second staging buffer while it
// transforms the current one, so HBM reads overlap the arithmetic.
#include "fit.h"
#include "regfft.cuh"

namespace fkk {
namespace {

struct KKWarpArgs {
  const float* i_cars;
  int64_t n;
  int m;
  int mpad;  // staging row length (m rounded up to 4)
  int64_t ld;
  const float* i_ref;
  float floor_;
  float* im;
  float* re;
  int64_t ld_out;
  long long* status;
  int vec16;  // rows are 16-byte aligned (16-byte cp.async)
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// rows 2 pr and 2 pr + 1 (if it exists) into the staging buffer
__device__ __forceinline__ void issue_pair(const KKWarpArgs& p, int64_t pr, float* st, int lane) {
  const int64_t n0 = 2 * pr;
  const int rows = (n0 + 1 < p.n) ? 2 : 1;
  for (int r = 0; r < rows; ++r) {
    const float* src = p.i_cars + (n0 + r) * p.ld;
    float* dst = st + r * p.mpad;
    int j0 = 0;
    if (p.vec16) {
      const int nv = p.m >> 2;
      for (int q = lane; q < nv; q += 32) cp_async16(dst + 4 * q, src + 4 * q);
      j0 = nv << 2;
    }
    for (int j = j0 + lane; j < p.m; j += 32) cp_async4(dst + j, src + j);
  }
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// slot of the 16-byte (PER = 2) or 8-byte (PER = 1) unit (row, c), c < 32
template <int PER>
__device__ __forceinline__ int slot(int row, int c) {
  return row * 32 + (c ^ (row & (PER == 2 ? 7 : 15)));
}

template <int R, bool kPhase>
__global__ void __launch_bounds__(R == 64 ? 192 : 384) kk_warp_kernel(KKWarpArgs p) {
  constexpr int L = 32 * R;
  constexpr int PER = R / 32;
  constexpr int LB = rf::ilog2(R);
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  // layout: twiddles (32 R float2) | 1/I_ref (mpad) | per warp: xbuf (L float2), stage[2] (2 mpad floats each)
  float2* tw = reinterpret_cast<float2*>(smem4);
  float* inv_ref = reinterpret_cast<float*>(tw + 32 * R);
  float2* wbase = reinterpret_cast<float2*>(inv_ref + p.mpad);
  const size_t per_warp_f2 = (size_t)L + 2 * (size_t)p.mpad;  // in float2 units
  float2* xbuf = wbase + wib * per_warp_f2;
  float* stage0 = reinterpret_cast<float*>(xbuf + L);
  const int M = p.m;
  const int left = (L - M) / 2;

  // w_L^(n1 k2), stored in the exchange layout: unit (n1, k2 / PER), element k2 % PER
  for (int e = threadIdx.x; e < 32 * R; e += blockDim.x) {
    const int n1 = e / R, k2 = e % R;
    float s, c;
    sincospif(-2.0f * (float)(n1 * k2) / (float)L, &s, &c);
    tw[slot<PER>(n1, k2 / PER) * PER + (k2 % PER)] = make_float2(c, s);
  }
  for (int j = threadIdx.x; j < M; j += blockDim.x) inv_ref[j] = 1.0f / p.i_ref[j];
  __syncthreads();

  const int64_t npairs = (p.n + 1) / 2;
  const int64_t nwarps = (int64_t)gridDim.x * nwb;
  int64_t pr = (int64_t)blockIdx.x * nwb + wib;
  int sbuf = 0;
  if (pr < npairs) issue_pair(p, pr, stage0, lane);
  cp_commit();
  int clamped = 0;
  constexpr float kL2eL = 1.4426950408889634f * (float)L;
  for (; pr < npairs; pr += nwarps) {
    const int64_t nx = pr + nwarps;
    float* st = stage0 + sbuf * 2 * p.mpad;
    if (nx < npairs) issue_pair(p, nx, stage0 + (sbuf ^ 1) * 2 * p.mpad, lane);
    cp_commit();
    cp_wait1();
    __syncwarp();
    const int64_t n0 = 2 * pr;
    const bool has1 = n0 + 1 < p.n;
    // a / L = (ln 2 / 2L) log2(max(I / I_ref, floor)) of both spectra, in
    // place (the 1/L of the inverse transform is folded in here, exactly:
    // L is a power of two)
    float* a0 = st;
    float* a1 = st + p.mpad;
    {
      const float cl = 0.34657359027997264f / (float)L;
      for (int j = lane; j < M; j += 32) {
        const float r = inv_ref[j];
        const float x0 = a0[j] * r;
        clamped += !(x0 >= p.floor_);
        a0[j] = cl * __log2f(fmaxf(x0, p.floor_));  // fmaxf takes the floor for NaN
        float v1 = 0.f;
        if (has1) {
          const float x1 = a1[j] * r;
          clamped += !(x1 >= p.floor_);
          v1 = cl * __log2f(fmaxf(x1, p.floor_));
        }
        a1[j] = v1;
      }
    }
    __syncwarp();
    float2 x[R];
    // edge-replicated, centred padding: z[t] = a[clamp(t - left)]
    rf::static_for<0, R>([&](auto q) {
      constexpr int n2 = decltype(q)::value;
      const int c = min(max(lane + 32 * n2 - left, 0), M - 1);
      x[n2] = make_float2(a0[c], a1[c]);
    });
    // ---- forward ----
    rf::fft_dif<R, -1>(x);  // x[i] = Y[n1][bitrev(i)]
    // twiddle and transpose out: unit (n1 = lane, c) holds k2 = PER c + b
    rf::static_for<0, 32>([&](auto q) {
      constexpr int c = decltype(q)::value;
      const int u = slot<PER>(lane, c);
      if constexpr (PER == 2) {
        constexpr int i0 = rf::bitrev(2 * c, LB), i1 = rf::bitrev(2 * c + 1, LB);
        const float4 t = reinterpret_cast<const float4*>(tw)[u];
        const float2 y0 = make_float2(fmaf(x[i0].x, t.x, -x[i0].y * t.y), fmaf(x[i0].x, t.y, x[i0].y * t.x));
        const float2 y1 = make_float2(fmaf(x[i1].x, t.z, -x[i1].y * t.w), fmaf(x[i1].x, t.w, x[i1].y * t.z));
        reinterpret_cast<float4*>(xbuf)[u] = make_float4(y0.x, y0.y, y1.x, y1.y);
      } else {
        constexpr int i0 = rf::bitrev(c, LB);
        const float2 t = tw[u];
        xbuf[u] = make_float2(fmaf(x[i0].x, t.x, -x[i0].y * t.y), fmaf(x[i0].x, t.y, x[i0].y * t.x));
      }
    });
    __syncwarp();
    // lane l: x[b*32 + n1] = Y'[n1][PER l + b]
    rf::static_for<0, 32>([&](auto q) {
      constexpr int n1 = decltype(q)::value;
      const int u = slot<PER>(n1, lane);
      if constexpr (PER == 2) {
        const float4 v = reinterpret_cast<const float4*>(xbuf)[u];
        x[n1] = make_float2(v.x, v.y);
        x[32 + n1] = make_float2(v.z, v.w);
      } else {
        x[n1] = xbuf[u];
      }
    });
    __syncwarp();
    rf::static_for<0, PER>([&](auto qb) {
      constexpr int b = decltype(qb)::value;
      rf::fft_dif<32, -1, b * 32>(x);  // x[b*32 + i] = X[k2 + R bitrev5(i)]
      const int k2 = PER * lane + b;
      // Hilbert multiplier -i sgn(k), k = k2 + R k1; 0 at DC and Nyquist
      rf::static_for<0, 32>([&](auto qi) {
        constexpr int i = decltype(qi)::value;
        constexpr int k1 = rf::bitrev(i, 5);
        float2& v = x[b * 32 + i];
        if constexpr (k1 == 0) {
          v = k2 == 0 ? make_float2(0.f, 0.f) : make_float2(v.y, -v.x);
        } else if constexpr (k1 < 16) {
          v = make_float2(v.y, -v.x);
        } else if constexpr (k1 == 16) {
          v = k2 == 0 ? make_float2(0.f, 0.f) : make_float2(-v.y, v.x);
        } else {
          v = make_float2(-v.y, v.x);
        }
      });
      rf::fft_dit<32, +1, b * 32>(x);  // x[b*32 + n1], natural n1
    });
    // conjugate twiddle and transpose back: unit (n1, lane)
    rf::static_for<0, 32>([&](auto q) {
      constexpr int n1 = decltype(q)::value;
      const int u = slot<PER>(n1, lane);
      if constexpr (PER == 2) {
        const float4 t = reinterpret_cast<const float4*>(tw)[u];
        const float2 a = x[n1], b = x[32 + n1];
        reinterpret_cast<float4*>(xbuf)[u] =
            make_float4(fmaf(a.x, t.x, a.y * t.y), fmaf(a.y, t.x, -a.x * t.y), fmaf(b.x, t.z, b.y * t.w),
                        fmaf(b.y, t.z, -b.x * t.w));
      } else {
        const float2 t = tw[u];
        const float2 a = x[n1];
        xbuf[u] = make_float2(fmaf(a.x, t.x, a.y * t.y), fmaf(a.y, t.x, -a.x * t.y));
      }
    });
    __syncwarp();
    rf::static_for<0, 32>([&](auto q) {
      constexpr int c = decltype(q)::value;
      const int u = slot<PER>(lane, c);
      if constexpr (PER == 2) {
        const float4 v = reinterpret_cast<const float4*>(xbuf)[u];
        x[2 * c] = make_float2(v.x, v.y);
        x[2 * c + 1] = make_float2(v.z, v.w);
      } else {
        x[c] = xbuf[u];
      }
    });
    rf::fft_dif<R, +1>(x);  // x[i] = h[lane + 32 bitrev(i)] (the input carried 1/L)
    // outputs: Im = e^a sin(phi), Re = e^a cos(phi) (or phi itself)
    float* im0 = p.im + n0 * p.ld_out;
    float* im1 = im0 + p.ld_out;
    rf::static_for<0, R>([&](auto q) {
      constexpr int i = decltype(q)::value;
      constexpr int n2 = rf::bitrev(i, LB);
      const int j = lane + 32 * n2 - left;
      if ((unsigned)j < (unsigned)M) {
        const float ph0 = x[i].x, ph1 = x[i].y;
        if (kPhase) {
          im0[j] = ph0;
          if (has1) im1[j] = ph1;
        } else {
          // e^a = 2^(a log2(e)); the stored value is a / L
          const float e0 = ex2_approx(kL2eL * a0[j]);
          im0[j] = e0 * __sinf(ph0);
          if (p.re) p.re[n0 * p.ld_out + j] = e0 * __cosf(ph0);
          if (has1) {
            const float e1 = ex2_approx(kL2eL * a1[j]);
            im1[j] = e1 * __sinf(ph1);
            if (p.re) p.re[(n0 + 1) * p.ld_out + j] = e1 * __cosf(ph1);
          }
        }
      }
    });
    __syncwarp();  // staging and exchange buffers are rewritten next
    sbuf ^= 1;
  }
  for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
  if (lane == 0 && clamped)
    atomicAdd(reinterpret_cast<unsigned long long*>(p.status + 1), (unsigned long long)clamped);
}

// ---------------------------------------------------------------------------
// Pad length 2,048 with four warps per pair of spectra (128 threads, 16
// complex values each) in three passes, n = a + 16 e + 128 f and
// k = g + 16 h + 128 d (a, g, f, d < 16; e, h < 8):
//   1. thread (a, e) = t holds samples t + 128 f: 16-point DFT over f,
//      twiddle w_128^(e g);
//   2. through shared memory to thread (a, g' = t / 16), which holds e for
//      g = g' and g' + 8: two 8-point DFTs over e, twiddle w_2048^(a c) with
//      c = g + 16 h;
//   3. through shared memory to thread c = t, which holds all a: 16-point
//      DFT over a -> X[c + 128 d];
// then -i sgn(k) in place and the same passes backwards.  Both exchanges
// use layouts that are conflict-free for the writer's and the reader's
// pattern, and the twiddle w_2048^(a c) is stored in the second layout.
// Sixteen values per thread (a two-warp form with 32 values per thread, 168
// registers, held twelve warps per SM and took 4.15 ms on 703,026 x 1,000;
// this one 3.20 ms) let six pairs (24 warps) share an SM.
__device__ __forceinline__ int qidx1(int a, int e, int g) { return g * 128 + e * 16 + a; }
__device__ __forceinline__ int qidx2(int a, int c) { return c * 16 + (a ^ (c & 15)); }

__device__ __forceinline__ void qbar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ float2 qmul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float2 qmulc(float2 a, float2 w) {  // a * conj(w)
  return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

constexpr int kQuadGroups = 6;

template <bool kPhase>
__global__ void __launch_bounds__(kQuadGroups * 128) kk_quad_kernel(KKWarpArgs p) {
  constexpr int L = 2048;
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31;
  const int grp = threadIdx.x >> 7, ngrp = blockDim.x >> 7;
  const int t = threadIdx.x & 127;
  const int ta = t & 15, tb = t >> 4;  // (a, e) in pass 1, (a, g') in pass 2, (g, h) in pass 3
  const int bar_id = 1 + grp;
  // layout: tw2 (2,048 float2, second exchange layout) | tw1 (128 float2) |
  //         1/I_ref (mpad) | per group: xbuf (2,048 float2), stage[2] (2 mpad floats each)
  float2* tw2 = reinterpret_cast<float2*>(smem4);
  float2* tw1 = tw2 + L;
  float* inv_ref = reinterpret_cast<float*>(tw1 + 128);
  float2* gbase = reinterpret_cast<float2*>(inv_ref + p.mpad);
  const size_t per_grp_f2 = (size_t)L + 2 * (size_t)p.mpad;
  float2* xbuf = gbase + grp * per_grp_f2;
  float* stage0 = reinterpret_cast<float*>(xbuf + L);
  const int M = p.m;
  const int left = (L - M) / 2;

  for (int q = threadIdx.x; q < L; q += blockDim.x) {
    const int a = q & 15, c = q >> 4;  // every (a, c) once
    float sv, cv;
    sincospif(-2.0f * (float)((a * c) & (L - 1)) / (float)L, &sv, &cv);
    tw2[qidx2(a, c)] = make_float2(cv, sv);
  }
  for (int q = threadIdx.x; q < 128; q += blockDim.x) {
    const int e = q >> 4, g = q & 15;
    float sv, cv;
    sincospif(-2.0f * (float)(e * g) / 128.0f, &sv, &cv);
    tw1[q] = make_float2(cv, sv);
  }
  for (int j = threadIdx.x; j < M; j += blockDim.x) inv_ref[j] = 1.0f / p.i_ref[j];
  __syncthreads();

  const int64_t npairs = (p.n + 1) / 2;
  const int64_t ngroups = (int64_t)gridDim.x * ngrp;
  int64_t pr = (int64_t)blockIdx.x * ngrp + grp;
  int sbuf = 0;
  // warps 0 and 1 of the group stage rows 0 and 1 of a pair
  const int wg = t >> 5;
  auto issue = [&](int64_t q, float* st) {
    if (wg > 1) return;
    const int64_t row = 2 * q + wg;
    if (row >= p.n) return;
    const float* src = p.i_cars + row * p.ld;
    float* dst = st + wg * p.mpad;
    int j0 = 0;
    if (p.vec16) {
      const int nv = M >> 2;
      for (int v = lane; v < nv; v += 32) cp_async16(dst + 4 * v, src + 4 * v);
      j0 = nv << 2;
    }
    for (int j = j0 + lane; j < M; j += 32) cp_async4(dst + j, src + j);
  };
  if (pr < npairs) issue(pr, stage0);
  cp_commit();
  int clamped = 0;
  constexpr float kL2eL = 1.4426950408889634f * (float)L;
  const float cl = 0.34657359027997264f / (float)L;
  for (; pr < npairs; pr += ngroups) {
    const int64_t nx = pr + ngroups;
    float* st = stage0 + sbuf * 2 * p.mpad;
    if (nx < npairs) issue(nx, stage0 + (sbuf ^ 1) * 2 * p.mpad);
    cp_commit();
    cp_wait1();
    qbar(bar_id);  // both rows staged
    const int64_t n0 = 2 * pr;
    const bool has1 = n0 + 1 < p.n;
    float* a0 = st;
    float* a1 = st + p.mpad;
    // a / L in place: (ln 2 / 2L) log2(max(I / I_ref, floor))
    for (int j = t; j < M; j += 128) {
      const float r = inv_ref[j];
      const float x0 = a0[j] * r;
      clamped += !(x0 >= p.floor_);
      a0[j] = cl * __log2f(fmaxf(x0, p.floor_));
      float v1 = 0.f;
      if (has1) {
        const float x1 = a1[j] * r;
        clamped += !(x1 >= p.floor_);
        v1 = cl * __log2f(fmaxf(x1, p.floor_));
      }
      a1[j] = v1;
    }
    qbar(bar_id);
    float2 x[16];
    // edge-replicated, centred padding: z[n] = a[clamp(n - left)], n = t + 128 f
    rf::static_for<0, 16>([&](auto q) {
      constexpr int f = decltype(q)::value;
      const int c = min(max(t + 128 * f - left, 0), M - 1);
      x[f] = make_float2(a0[c], a1[c]);
    });
    // ---- forward ----
    rf::fft_dif<16, -1>(x);  // x[i] = Z[g = bitrev(i)]
    rf::static_for<0, 16>([&](auto q) {
      constexpr int i = decltype(q)::value;
      constexpr int g = rf::bitrev(i, 4);
      xbuf[qidx1(ta, tb, g)] = qmul(x[i], tw1[tb * 16 + g]);
    });
    qbar(bar_id);
    rf::static_for<0, 16>([&](auto q) {  // x[8 s + e] for g = tb + 8 s
      constexpr int i = decltype(q)::value;
      x[i] = xbuf[qidx1(ta, i & 7, tb + 8 * (i >> 3))];
    });
    rf::fft_dif<8, -1, 0>(x);
    rf::fft_dif<8, -1, 8>(x);  // x[8 s + i'] = Y[c = tb + 8 s + 16 bitrev3(i')]
    qbar(bar_id);              // every thread has read the first exchange
    rf::static_for<0, 16>([&](auto q) {
      constexpr int i = decltype(q)::value;
      const int c = tb + 8 * (i >> 3) + 16 * rf::bitrev(i & 7, 3);
      const int u = qidx2(ta, c);
      xbuf[u] = qmul(x[i], tw2[u]);
    });
    qbar(bar_id);
    rf::static_for<0, 16>([&](auto q) {
      constexpr int a = decltype(q)::value;
      x[a] = xbuf[qidx2(a, t)];
    });
    rf::fft_dif<16, -1>(x);  // x[i] = X[t + 128 d], d = bitrev(i)
    // -i sgn(k), k = t + 128 d: d < 8 below L/2; DC (t = 0, d = 0) and Nyquist (t = 0, d = 8) vanish
    rf::static_for<0, 16>([&](auto q) {
      constexpr int i = decltype(q)::value;
      constexpr int d = rf::bitrev(i, 4);
      const float2 v = x[i];
      float2 r = d < 8 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
      if (d == 0 || d == 8) r = t == 0 ? make_float2(0.f, 0.f) : r;
      x[i] = r;
    });
    // ---- inverse ----
    rf::fft_dit<16, +1>(x);  // x[a], natural
    qbar(bar_id);            // every thread has read the second exchange
    rf::static_for<0, 16>([&](auto q) {
      constexpr int a = decltype(q)::value;
      const int u = qidx2(a, t);
      xbuf[u] = qmulc(x[a], tw2[u]);
    });
    qbar(bar_id);
    rf::static_for<0, 16>([&](auto q) {  // bit-reversed h for the DIT passes
      constexpr int i = decltype(q)::value;
      const int c = tb + 8 * (i >> 3) + 16 * rf::bitrev(i & 7, 3);
      x[i] = xbuf[qidx2(ta, c)];
    });
    rf::fft_dit<8, +1, 0>(x);
    rf::fft_dit<8, +1, 8>(x);  // x[8 s + e]
    qbar(bar_id);
    rf::static_for<0, 16>([&](auto q) {
      constexpr int i = decltype(q)::value;
      const int g = tb + 8 * (i >> 3);
      xbuf[qidx1(ta, i & 7, g)] = qmulc(x[i], tw1[(i & 7) * 16 + g]);
    });
    qbar(bar_id);
    rf::static_for<0, 16>([&](auto q) {  // bit-reversed g
      constexpr int i = decltype(q)::value;
      x[i] = xbuf[qidx1(ta, tb, rf::bitrev(i, 4))];
    });
    rf::fft_dit<16, +1>(x);  // x[f]: sample t + 128 f of H{a0} + i H{a1}
    float* im0 = p.im + n0 * p.ld_out;
    float* im1 = im0 + p.ld_out;
    rf::static_for<0, 16>([&](auto q) {
      constexpr int f = decltype(q)::value;
      const int j = t + 128 * f - left;
      if ((unsigned)j < (unsigned)M) {
        const float ph0 = x[f].x, ph1 = x[f].y;
        if (kPhase) {
          im0[j] = ph0;
          if (has1) im1[j] = ph1;
        } else {
          const float e0 = ex2_approx(kL2eL * a0[j]);
          im0[j] = e0 * __sinf(ph0);
          if (p.re) p.re[n0 * p.ld_out + j] = e0 * __cosf(ph0);
          if (has1) {
            const float e1 = ex2_approx(kL2eL * a1[j]);
            im1[j] = e1 * __sinf(ph1);
            if (p.re) p.re[(n0 + 1) * p.ld_out + j] = e1 * __cosf(ph1);
          }
        }
      }
    });
    qbar(bar_id);  // staging and exchange buffers are rewritten next
    sbuf ^= 1;
  }
  for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
  if (lane == 0 && clamped)
    atomicAdd(reinterpret_cast<unsigned long long*>(p.status + 1), (unsigned long long)clamped);
}

template <bool kPhase>
fkk_status launch_quad(fkk_ctx* ctx, const KKWarpArgs& a, cudaStream_t st) {
  const size_t fixed = sizeof(float2) * (2048 + 128) + sizeof(float) * (size_t)a.mpad;
  const size_t pg = sizeof(float2) * (2048 + 2 * (size_t)a.mpad);
  const size_t cap = 227 * 1024;
  int groups = kQuadGroups;
  while (groups > 1 && fixed + groups * pg > cap) --groups;
  const size_t smem = fixed + groups * pg;
  if (smem > cap) return fail(ctx, FKK_ERR_INVALID_ARG, "kk: %d channels need %zu B of shared memory", a.m, smem);
  auto fn = kk_quad_kernel<kPhase>;
  FKK_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t npairs = (a.n + 1) / 2;
  int64_t grid = (npairs + groups - 1) / groups;
  grid = std::min<int64_t>(grid, ctx->sm_count);
  if (grid < 1) grid = 1;
  FKK_COUNT_LAUNCH();
  fn<<<(unsigned)grid, groups * 128, smem, st>>>(a);
  return cuda_check(ctx, cudaGetLastError(), "kk_quad_kernel launch");
}

template <int R>
size_t kk_warp_fixed_smem(int mpad) {
  return sizeof(float2) * 32 * (size_t)R + sizeof(float) * (size_t)mpad;
}
template <int R>
size_t kk_warp_per_warp(int mpad) {
  return sizeof(float2) * (32 * (size_t)R + 2 * (size_t)mpad);
}

template <int R, bool kPhase>
fkk_status launch_r(fkk_ctx* ctx, const KKWarpArgs& a, cudaStream_t st) {
  const size_t fixed = kk_warp_fixed_smem<R>(a.mpad), pw = kk_warp_per_warp<R>(a.mpad);
  const size_t cap = 227 * 1024;
  int warps = R == 64 ? 6 : 12;
  while (warps > 1 && fixed + warps * pw > cap) --warps;
  const size_t smem = fixed + warps * pw;
  if (smem > cap) return fail(ctx, FKK_ERR_INVALID_ARG, "kk: %d channels need %zu B of shared memory", a.m, smem);
  auto fn = kk_warp_kernel<R, kPhase>;
  FKK_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t npairs = (a.n + 1) / 2;
  int64_t grid = (npairs + warps - 1) / warps;
  grid = std::min<int64_t>(grid, ctx->sm_count);
  if (grid < 1) grid = 1;
  FKK_COUNT_LAUNCH();
  fn<<<(unsigned)grid, warps * 32, smem, st>>>(a);
  return cuda_check(ctx, cudaGetLastError(), "kk_warp_kernel launch");
}

}  // namespace

// The register-FFT form handles L = 1024 and 2048 with m <= L; returns
// FKK_ERR_INVALID_ARG with *handled = false for other lengths.
fkk_status launch_kk_warp(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld, const float* i_ref,
                          int L, float floor_, float* im, float* re, int64_t ld_out, bool phase, cudaStream_t st,
                          bool* handled) {
  *handled = false;
  if (L != 1024 && L != 2048) return FKK_OK;
  if (m > L) return FKK_OK;
  KKWarpArgs a{};
  a.i_cars = i_cars;
  a.n = n;
  a.m = m;
  a.mpad = (m + 3) & ~3;
  a.ld = ld;
  a.i_ref = i_ref;
  a.floor_ = floor_;
  a.im = im;
  a.re = phase ? nullptr : re;
  a.ld_out = ld_out;
  a.status = ctx->d_status;
  a.vec16 = ((reinterpret_cast<uintptr_t>(i_cars) & 15) == 0) && (ld % 4 == 0);
  *handled = true;
  if (L == 2048) return phase ? launch_quad<true>(ctx, a, st) : launch_quad<false>(ctx, a, st);
  return phase ? launch_r<32, true>(ctx, a, st) : launch_r<32, false>(ctx, a, st);
}

}  // namespace fkk
