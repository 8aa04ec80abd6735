// Per-spectrum KK (Eq. KCARS with the surrogate reference of Eq. K) with one
// warp per pair of spectra and the length-L transform held in registers.
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
  const float invL = 1.0f / (float)L;
  for (; pr < npairs; pr += nwarps) {
    const int64_t nx = pr + nwarps;
    float* st = stage0 + sbuf * 2 * p.mpad;
    if (nx < npairs) issue_pair(p, nx, stage0 + (sbuf ^ 1) * 2 * p.mpad, lane);
    cp_commit();
    cp_wait1();
    __syncwarp();
    const int64_t n0 = 2 * pr;
    const bool has1 = n0 + 1 < p.n;
    float* a0 = st;
    float* a1 = st + p.mpad;
    // a = 1/2 ln(max(I / I_ref, floor)), in place
    for (int j = lane; j < M; j += 32) {
      const float r = inv_ref[j];
      float x0 = a0[j] * r;
      if (!(x0 >= p.floor_)) { x0 = p.floor_; ++clamped; }
      a0[j] = 0.34657359027997264f * __log2f(x0);  // (ln 2 / 2) log2
      float v1 = 0.f;
      if (has1) {
        float x1 = a1[j] * r;
        if (!(x1 >= p.floor_)) { x1 = p.floor_; ++clamped; }
        v1 = 0.34657359027997264f * __log2f(x1);
      }
      a1[j] = v1;
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
    rf::fft_dif<R, +1>(x);  // x[i] = L h[lane + 32 bitrev(i)]
    // outputs: Im = e^a sin(phi), Re = e^a cos(phi) (or phi itself)
    float* im0 = p.im + n0 * p.ld_out;
    float* im1 = im0 + p.ld_out;
    rf::static_for<0, R>([&](auto q) {
      constexpr int i = decltype(q)::value;
      constexpr int n2 = rf::bitrev(i, LB);
      const int j = lane + 32 * n2 - left;
      if ((unsigned)j < (unsigned)M) {
        const float ph0 = x[i].x * invL, ph1 = x[i].y * invL;
        if (kPhase) {
          im0[j] = ph0;
          if (has1) im1[j] = ph1;
        } else {
          const float e0 = exp2f(1.4426950408889634f * a0[j]);
          im0[j] = e0 * __sinf(ph0);
          if (p.re) p.re[n0 * p.ld_out + j] = e0 * __cosf(ph0);
          if (has1) {
            const float e1 = exp2f(1.4426950408889634f * a1[j]);
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
  if (L == 2048) return phase ? launch_r<64, true>(ctx, a, st) : launch_r<64, false>(ctx, a, st);
  return phase ? launch_r<32, true>(ctx, a, st) : launch_r<32, false>(ctx, a, st);
}

}  // namespace fkk
