// The conventional per-spectrum workflow (Sec. 2.1 and Fig. 1(a);
// Eq. KCARS_from_K), the baseline the factorised method is measured against:
//   X       <- X_k, the truncated SVD of the raw spectra        (optional)
//   a       = 1/2 ln max(I/I_ref, floor),  phi = H{a}              (Eq. K)
//   phi_err = D{phi}, the asymmetric-least-squares baseline         (PEC)
//   K_pec   = exp(a + H{phi_err}) exp(i (phi - phi_err))
//   K_CARS  = K_pec / M{Re K_pec}, M the trendline (or the mean)    (SEC)
//
// Spectra are processed in chunks.  Per chunk:
//   1. the paired-FFT KK kernel in its phase mode writes phi (row-major);
//   2. als_kernel runs the detrend with one thread per spectrum: each of the
//      reweighting iterations solves (W + lam D2^T D2) z = W y, a symmetric
//      pentadiagonal system, by a banded LDL^T forward sweep (storing the
//      factor columns l1, l2 and D^-1 L^-1 W y) and a backward sweep (which
//      also records the new weights as bits).  The system's condition number
//      reaches 1e7 (lam up to ~1e5 against weights of 1e-2), so the solves run
//      in double-word arithmetic; the 32 spectra of a warp go through shared
//      memory tiles so that every global access of the sweeps is coalesced;
//   3. conv_finish_kernel forms H{phi_err} (paired FFT), K_pec and the
//      trendline of Re K_pec per spectrum -- Savitzky-Golay of order <= 2 as
//      the correlation with the centre-value kernel by a second paired FFT,
//      with the first / last full window's polynomial at the edges; or the
//      mean -- and writes Im (and Re) K_CARS.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "df64.cuh"
#include "fft.cuh"
#include "fit.h"
#include "fkk_internal.h"

namespace fkk {
namespace {

using dw::df;

// ------------------------------------------------------------------- ALS ---

constexpr int kAlsThreads = 128;
constexpr int kAlsWarps = kAlsThreads / 32;

struct AlsArgs {
  const float* phi;  // n x m row-major (row stride m): the signal y of each spectrum
  float* perr;       // n x m row-major: the baseline z of the last iteration
  float2* fac;       // [m][3][ns]: l1, l2, h (double-word) of the forward sweep
  unsigned* bits;    // [ceil(m/32)][ns]: bit r of word b = (y > z) at row 32 b + r
  int64_t n;         // spectra
  int64_t ns;        // interleave stride: >= n, a multiple of 32
  int m;
  double lam, p;
  int iters;
};

// Coefficients of D2^T D2 (D2 the (m-2) x m second-difference operator):
// diagonal 1, 5, 6, ..., 6, 5, 1 and first off-diagonal -2, -4, ..., -4, -2
// (general m >= 3); the second off-diagonal is 1.
__device__ __forceinline__ float dtd0(int i, int m) {
  return (i <= m - 3 ? 1.f : 0.f) + (i >= 1 && i <= m - 2 ? 4.f : 0.f) + (i >= 2 ? 1.f : 0.f);
}
__device__ __forceinline__ float dtd1(int i, int m) {  // entry (i, i+1)
  return (i <= m - 3 ? -2.f : 0.f) + (i >= 1 && i <= m - 2 ? -2.f : 0.f);
}

__global__ void __launch_bounds__(kAlsThreads, 8) als_kernel(AlsArgs a) {
  __shared__ float tiles[kAlsWarps][32][33];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kAlsThreads + wib * 32;  // the warp's first spectrum
  if (base >= a.n) return;  // no block-wide barrier below: a warp may leave
  float(*T)[33] = tiles[wib];
  const int64_t s = base + lane;
  const bool live = s < a.n;
  const int m = a.m, nblk = (m + 31) / 32;
  const int64_t ns = a.ns;
  const df lam = dw::from_double(a.lam);
  const df pw = dw::from_double(a.p), qw = dw::from_double(1.0 - a.p), one = dw::make(1.f);

  // T[q][r] = y of spectrum base + q at row 32 rb + r (0 outside)
  auto load_tile = [&](int rb) {
    __syncwarp();
    const int i = rb * 32 + lane;
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      const int64_t sq = base + q;
      T[q][lane] = (sq < a.n && i < m) ? __ldg(a.phi + sq * m + i) : 0.f;
    }
    __syncwarp();
  };

  for (int it = 0; it < a.iters; ++it) {
    const bool last = it == a.iters - 1;
    // forward: L D L^T = W + lam D2^T D2 and g = L^-1 W y, one row at a time.
    // With c_i = l1_i d_{i-1}: l2_i = lam / d_{i-2}, c_i = lam t1_{i-1} -
    // l2_i c_{i-1}, l1_i = c_i / d_{i-1}, d_i = w_i + lam t0_i - l1_i c_i -
    // l2_i lam, g_i = w_i y_i - l1_i g_{i-1} - l2_i g_{i-2}.
    df rd1 = dw::make(0.f), rd2 = dw::make(0.f), c1 = dw::make(0.f), g1 = dw::make(0.f), g2 = dw::make(0.f);
    for (int rb = 0; rb < nblk; ++rb) {
      load_tile(rb);
      const unsigned wb = (it > 0 && live) ? a.bits[(int64_t)rb * ns + s] : 0u;
      const int rows = min(32, m - rb * 32);
#pragma unroll 1
      for (int r = 0; r < rows; ++r) {
        const int i = rb * 32 + r;
        const float y = T[lane][r];
        const df w = it == 0 ? one : (((wb >> r) & 1u) ? pw : qw);
        const df l2 = i >= 2 ? dw::mul(lam, rd2) : dw::make(0.f);
        df c = dw::make(0.f), l1 = dw::make(0.f);
        if (i >= 1) {
          c = dw::sub(dw::mul(lam, dtd1(i - 1, m)), dw::mul(l2, c1));
          l1 = dw::mul(c, rd1);
        }
        const df d = dw::sub(dw::sub(dw::add(w, dw::mul(lam, dtd0(i, m))), dw::mul(l1, c)), dw::mul(l2, lam));
        const df g = dw::sub(dw::sub(dw::mul(w, y), dw::mul(l1, g1)), dw::mul(l2, g2));
        const df rd = dw::rcp(d);
        const df h = dw::mul(g, rd);
        if (live) {
          float2* f = a.fac + (int64_t)i * 3 * ns + s;
          f[0] = make_float2(l1.h, l1.l);
          f[ns] = make_float2(l2.h, l2.l);
          f[2 * ns] = make_float2(h.h, h.l);
        }
        rd2 = rd1;
        rd1 = rd;
        c1 = c;
        g2 = g1;
        g1 = g;
      }
    }
    // backward: z_i = h_i - l1_{i+1} z_{i+1} - l2_{i+2} z_{i+2}; the next
    // weights are p where y > z, else 1 - p
    df z1 = dw::make(0.f), z2 = dw::make(0.f), l1n = dw::make(0.f), l2n1 = dw::make(0.f), l2n2 = dw::make(0.f);
    for (int rb = nblk - 1; rb >= 0; --rb) {
      load_tile(rb);
      unsigned wb = 0;
      const int rows = min(32, m - rb * 32);
#pragma unroll 1
      for (int r = rows - 1; r >= 0; --r) {
        const int i = rb * 32 + r;
        df l1 = dw::make(0.f), l2 = dw::make(0.f), h = dw::make(0.f);
        if (live) {
          const float2* f = a.fac + (int64_t)i * 3 * ns + s;
          const float2 f0 = f[0], f1 = f[ns], f2 = f[2 * ns];
          l1 = dw::make(f0.x, f0.y);
          l2 = dw::make(f1.x, f1.y);
          h = dw::make(f2.x, f2.y);
        }
        const df z = dw::sub(dw::sub(h, dw::mul(l1n, z1)), dw::mul(l2n2, z2));
        const float y = T[lane][r];
        const df dyz = dw::sub(dw::make(y), z);
        if (dyz.h > 0.f || (dyz.h == 0.f && dyz.l > 0.f)) wb |= 1u << r;
        if (last) T[lane][r] = z.h + z.l;
        l2n2 = l2n1;
        l2n1 = l2;
        l1n = l1;
        z2 = z1;
        z1 = z;
      }
      if (!last) {
        if (live) a.bits[(int64_t)rb * ns + s] = wb;
      } else {
        __syncwarp();
        const int i = rb * 32 + lane;
        if (i < m)
          for (int q = 0; q < 32; ++q) {
            const int64_t sq = base + q;
            if (sq < a.n) a.perr[sq * m + i] = T[q][lane];
          }
      }
    }
  }
}

// ---------------------------------------------------------------- finish ---

constexpr int kFinThreads = 256;
constexpr int kFinWarps = kFinThreads / 32;

struct FinArgs {
  const float* i_cars;
  int64_t ld;
  const float* i_ref;
  const float* phi;   // n x m, row stride m
  const float* perr;  // n x m, row stride m (null: no PEC)
  const float* sgk;   // L: DFT of the Savitzky-Golay centre-value kernel (real)
  int64_t n;
  int m, L;
  float floor_;
  int sec;            // 0 off, 1 Savitzky-Golay, 2 mean
  int window;         // odd Savitzky-Golay window
  float gi[9];        // inverse of the window's moment matrix sum_t t^(a+b), a, b <= order
  float* im;
  float* re;
  int64_t ld_out;
};

// Sums v[0..11] over the tpf threads of a slot (whole warps); every thread
// of the slot gets the totals.  red: kFinWarps * 12 floats per slot.
// Block-wide barriers.
__device__ void slot_sum12(float (&v)[12], int t0, int tpf, float* red) {
#pragma unroll
  for (int q = 0; q < 12; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((t0 & 31) == 0)
#pragma unroll
    for (int q = 0; q < 12; ++q) red[(t0 >> 5) * 12 + q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    float t = 0.f;
    for (int w = 0; w < tpf / 32; ++w) t += red[w * 12 + q];
    v[q] = t;
  }
  __syncthreads();
}

// The fitted polynomial of a window at offset u from its centre, from the
// window's moments m0..m2 about that centre.
__device__ __forceinline__ float window_value(const float* gi, float m0, float m1, float m2, float u) {
  const float c0 = gi[0] * m0 + gi[1] * m1 + gi[2] * m2;
  const float c1 = gi[3] * m0 + gi[4] * m1 + gi[5] * m2;
  const float c2 = gi[6] * m0 + gi[7] * m1 + gi[8] * m2;
  return c0 + u * (c1 + u * c2);
}

__global__ void __launch_bounds__(kFinThreads) conv_finish_kernel(FinArgs p, int tpf) {
  extern __shared__ float4 smem_raw[];
  const int L = p.L, M = p.m;
  const int nfft = blockDim.x / tpf, f = threadIdx.x / tpf, t0 = threadIdx.x % tpf;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* buf0 = tw + L + f * (2 * L);
  float2* buf1 = buf0 + L;
  float* fbase = reinterpret_cast<float*>(tw + L + nfft * 2 * L);
  float* sre = fbase + (size_t)f * 4 * M;  // Re K_pec of the two spectra, then Im
  float* sim = sre + 2 * M;
  float* red = fbase + (size_t)nfft * 4 * M + f * kFinWarps * 12;
  const int left = (L - M) / 2;
  const float invL = 1.0f / (float)L;
  const int W = p.window, hw = W / 2;

  fill_twiddles(tw, L);
  const int64_t npairs = (p.n + 1) / 2;
  for (int64_t bp = (int64_t)blockIdx.x * nfft; bp < npairs; bp += (int64_t)gridDim.x * nfft) {
    __syncthreads();
    const int64_t pr = bp + f;
    const bool live = pr < npairs;
    const int64_t n0 = 2 * pr, n1 = 2 * pr + 1;
    const bool has1 = live && n1 < p.n;
    // H{phi_err} of both spectra (one complex FFT)
    const float2* hb = nullptr;
    if (p.perr) {
      for (int t = t0; t < L; t += tpf) {
        const int j = min(max(t - left, 0), M - 1);
        buf0[t] = make_float2(live ? p.perr[n0 * M + j] : 0.f, has1 ? p.perr[n1 * M + j] : 0.f);
      }
      __syncthreads();
      const int cur = fft_block<-1>(buf0, buf1, L, tw, t0, tpf);
      float2* X = cur ? buf1 : buf0;
      float2* Y = cur ? buf0 : buf1;
      for (int t = t0; t < L; t += tpf) X[t] = hilbert_mult(X[t], t, L);
      __syncthreads();
      const int cur2 = fft_block<+1>(X, Y, L, tw, t0, tpf);
      hb = cur2 ? Y : X;
    }
    // K_pec of both spectra
    for (int j = t0; j < M; j += tpf) {
      const float r = 1.0f / p.i_ref[j];
      for (int q = 0; q < 2; ++q) {
        const bool ok = q == 0 ? live : has1;
        float re = 0.f, im = 0.f;
        if (ok) {
          const int64_t nq = q == 0 ? n0 : n1;
          float x = p.i_cars[nq * p.ld + j] * r;
          if (!(x >= p.floor_)) x = p.floor_;
          const float av = 0.34657359027997264f * __log2f(x);  // as kk_per_spectrum
          float hv = 0.f, pe = 0.f;
          if (p.perr) {
            const float2 hh = hb[left + j];
            hv = (q == 0 ? hh.x : hh.y) * invL;
            pe = p.perr[nq * M + j];
          }
          const float amp = exp2f(1.4426950408889634f * (av + hv));
          const float ph = p.phi[nq * M + j] - pe;
          const float sn = __sinf(ph), cs = __cosf(ph);
          re = amp * cs;
          im = amp * sn;
        }
        sre[q * M + j] = re;
        sim[q * M + j] = im;
      }
    }
    __syncthreads();
    // SEC: the trendline of Re K_pec.  Savitzky-Golay: the centre values are
    // the correlation of Re K_pec with the centre-value kernel (an FFT pair,
    // the two spectra in one complex transform, zero-padded so nothing
    // wraps); near the edges, the polynomial of the first / last full window
    // from its three moments.  Mean: the channel sum.
    float mom[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) mom[q] = 0.f;
    const float2* cb = nullptr;
    if (p.sec == 1) {
      for (int t = t0; t < L; t += tpf) buf0[t] = t < M ? make_float2(sre[t], sre[M + t]) : make_float2(0.f, 0.f);
      for (int i = t0; i < W; i += tpf) {
        const float u = (float)(i - hw);
        const float xl0 = sre[i], xl1 = sre[M + i];
        const float xh0 = sre[M - W + i], xh1 = sre[2 * M - W + i];
        mom[0] += xl0;
        mom[1] += u * xl0;
        mom[2] += u * u * xl0;
        mom[3] += xh0;
        mom[4] += u * xh0;
        mom[5] += u * u * xh0;
        mom[6] += xl1;
        mom[7] += u * xl1;
        mom[8] += u * u * xl1;
        mom[9] += xh1;
        mom[10] += u * xh1;
        mom[11] += u * u * xh1;
      }
      __syncthreads();
      const int cur = fft_block<-1>(buf0, buf1, L, tw, t0, tpf);
      float2* X = cur ? buf1 : buf0;
      float2* Y = cur ? buf0 : buf1;
      for (int t = t0; t < L; t += tpf) {
        const float k = p.sgk[t];
        X[t] = make_float2(X[t].x * k, X[t].y * k);
      }
      __syncthreads();
      const int cur2 = fft_block<+1>(X, Y, L, tw, t0, tpf);
      cb = cur2 ? Y : X;
    } else if (p.sec == 2) {
      for (int j = t0; j < M; j += tpf) {
        mom[0] += sre[j];
        mom[6] += sre[M + j];
      }
    }
    if (p.sec) slot_sum12(mom, t0, tpf, red);
    for (int q = 0; q < 2; ++q) {
      const bool ok = q == 0 ? live : has1;
      if (!ok) continue;
      const int64_t nq = q == 0 ? n0 : n1;
      const float* mq = mom + 6 * q;
      for (int j = t0; j < M; j += tpf) {
        float tr = 1.f;
        if (p.sec == 2) {
          tr = mq[0] / (float)M;
        } else if (p.sec == 1) {
          if (j < hw) tr = window_value(p.gi, mq[0], mq[1], mq[2], (float)(j - hw));
          else if (j >= M - hw) tr = window_value(p.gi, mq[3], mq[4], mq[5], (float)(j - (M - 1 - hw)));
          else tr = (q == 0 ? cb[j].x : cb[j].y) * invL;
        }
        const float inv = 1.f / tr;
        p.im[nq * p.ld_out + j] = sim[q * M + j] * inv;
        if (p.re) p.re[nq * p.ld_out + j] = sre[q * M + j] * inv;
      }
    }
  }
}

// DFT (length L) of the even Savitzky-Golay centre-value kernel
// k(t) = g00 + g01 t + g02 t^2 on |t| <= h (zero elsewhere, t taken mod L).
__global__ void sg_kernel_dft_kernel(int L, int h, double g00, double g01, double g02, float* out) {
  const int mq = blockIdx.x * blockDim.x + threadIdx.x;
  if (mq >= L) return;
  double acc = 0.0;
  for (int t = -h; t <= h; ++t) {
    const long long mt = ((long long)mq * (t + L)) % L;
    acc += (g00 + t * (g01 + t * g02)) * cospi(2.0 * (double)mt / (double)L);
  }
  out[mq] = (float)acc;
}

// inverse of the (order+1) x (order+1) moment matrix of the window
// t = -h..h, embedded in a 3 x 3 array (zeros beyond the order)
bool window_moment_inverse(int window, int order, double* gi) {
  const int h = window / 2, n = order + 1;
  double g[3][6] = {};
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int t = -h; t <= h; ++t) s += std::pow((double)t, r + c);
      g[r][c] = s;
    }
    g[r][n + r] = 1.0;
  }
  for (int c = 0; c < n; ++c) {  // Gauss-Jordan with partial pivoting
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(g[r][c]) > std::fabs(g[piv][c])) piv = r;
    if (g[piv][c] == 0.0) return false;
    for (int k = 0; k < 2 * n; ++k) std::swap(g[c][k], g[piv][k]);
    const double d = g[c][c];
    for (int k = 0; k < 2 * n; ++k) g[c][k] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const double e = g[r][c];
        for (int k = 0; k < 2 * n; ++k) g[r][k] -= e * g[c][k];
      }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gi[3 * r + c] = (r < n && c < n) ? g[r][n + c] : 0.0;
  return true;
}

size_t finish_smem_bytes(int L, int M, int nfft) {
  return sizeof(float2) * (size_t)L + (size_t)nfft * (2 * L * sizeof(float2) + 4 * M * sizeof(float)) +
         (size_t)nfft * kFinWarps * 12 * sizeof(float);
}


// Vt (k x m) = V^T for V (m x k, row stride ldv).
__global__ void transpose_v_kernel(const double* __restrict__ v, int m, int k, int ldv, double* __restrict__ vt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * k) return;
  const int i = (int)(t / m), j = (int)(t % m);
  vt[t] = v[(int64_t)j * ldv + i];
}

// b = V V^T c (m), one block: the shift's share of X_k = (D + 1 c^T) V V^T.
__global__ void shift_share_kernel(const double* __restrict__ v, const float* __restrict__ c, int m, int k,
                                   float* __restrict__ b) {
  __shared__ double t[80];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = w; i < k; i += nw) {
    double acc = 0.0;
    for (int j = lane; j < m; j += 32) acc += (double)c[j] * v[(int64_t)j * k + i];
    acc = warp_sum(acc);
    if (lane == 0) t[i] = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += v[(int64_t)j * k + i] * t[i];
    b[j] = (float)acc;
  }
}

// The conventional workflow's denoising step (Fig. 1(a); Sec. 2.2): the
// truncated SVD X_k = (X V_k) V_k^T of the raw spectra X (n x m), V_k the k
// leading eigenvectors of X^T X.  The Gram matrix, the eigensolver, the
// projection and the reconstruction are the fit's kernels, the transform in
// its raw mode (D = X - 1 c^T) and the reconstruction with its linear
// epilogue.  Raw spectra are dominated by their mean, so the tensor cores
// see only D: X_k = (D V_k) V_k^T + 1 (V_k V_k^T c)^T, the second term
// exact in fp64 and added per channel.
// *out: n x m (row stride m) in the context's workspace.
fkk_status svd_denoise(fkk_ctx* ctx, const float* x, int64_t n, int m, int64_t ld, const fkk_fit_params& pp,
                       float** out, cudaStream_t st) {
  fkk_status s;
  DtLayout D;
  FKK_TRY(launch_transform(ctx, x, n, m, ld, nullptr, 0.f, D, st, true));
  double* G = (double*)workspace(ctx, "dn_gram", (size_t)m * m * 8, &s);
  if (!G) return s;
  FKK_TRY(launch_gram(ctx, D, nullptr, G, st));
  const bool rule = pp.denoise_k < 0;
  const int ke = rule ? std::min(pp.k_max, m) : pp.denoise_k;  // eigenpairs computed
  double* lam = (double*)workspace(ctx, "dn_lam", (size_t)ke * 8, &s);
  if (!lam) return s;
  double* v = (double*)workspace(ctx, "dn_v", (size_t)m * ke * 8, &s);
  if (!v) return s;
  FKK_TRY(launch_eig_topk(ctx, G, m, ke, lam, v, st));
  int k = ke;
  if (rule) {  // the rank rule of Sec. 4.1, as fkk_fit_basis applies it
    std::vector<double> lh(ke);
    FKK_CUDA(ctx, cudaMemcpyAsync(lh.data(), lam, (size_t)ke * 8, cudaMemcpyDeviceToHost, st));
    FKK_CUDA(ctx, cudaStreamSynchronize(st));
    const double eps = pp.rank_eps > 0.0 ? pp.rank_eps : (double)FLT_EPSILON;
    const double tol = std::sqrt(std::max(lh[0], 0.0)) * (double)std::max<int64_t>(n, m) * eps;
    k = 0;
    while (k < ke && std::sqrt(std::max(lh[k], 0.0)) > tol) ++k;
    if (k < 1) k = 1;
  }
  double* vk = v;
  if (k < ke) {  // the projection reads V_k with row stride k
    vk = (double*)workspace(ctx, "dn_vk", (size_t)m * k * 8, &s);
    if (!vk) return s;
    FKK_CUDA(ctx, cudaMemcpy2DAsync(vk, (size_t)k * 8, v, (size_t)ke * 8, (size_t)k * 8, m, cudaMemcpyDeviceToDevice, st));
  }
  float* P = (float*)workspace(ctx, "dn_p", (size_t)n * k * 4, &s);
  if (!P) return s;
  DtLayout Dv = D;
  Dv.c = nullptr;  // P = D V_k, without the shift's offset
  FKK_TRY(launch_project(ctx, Dv, vk, nullptr, k, P, nullptr, nullptr, st));
  float* b = (float*)workspace(ctx, "dn_bias", (size_t)m * 4, &s);
  if (!b) return s;
  FKK_COUNT_LAUNCH(); shift_share_kernel<<<1, 256, 0, st>>>(vk, D.c, m, k, b);
  double* vt = (double*)workspace(ctx, "dn_vt", (size_t)m * k * 8, &s);
  if (!vt) return s;
  const int64_t tot = (int64_t)m * k;
  FKK_COUNT_LAUNCH(); transpose_v_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(vk, m, k, k, vt);
  FKK_CUDA(ctx, cudaGetLastError());
  float* xk = (float*)workspace(ctx, "dn_out", (size_t)n * m * 4, &s);
  if (!xk) return s;
  FKK_TRY(launch_reconstruct_linear(ctx, P, n, k, m, vt, b, xk, m, st));
  *out = xk;
  return FKK_OK;
}

}  // namespace
}  // namespace fkk

using namespace fkk;

extern "C" fkk_status conventional_per_spectrum(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra,
                                                int32_t n_channels, int64_t ld, const float* i_ref,
                                                const fkk_fit_params* params, float* im_out, float* re_out,
                                                int64_t ld_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const int m = n_channels;
  if (!params || n_spectra < 0 || m < 8 || m > 2048 || ld < m || ld_out < m)
    return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: bad sizes (n=%lld m=%d)", (long long)n_spectra, m);
  const fkk_fit_params& pp = *params;
  const int L = pp.pad_len ? pp.pad_len : next_pow2(2 * (int64_t)m);
  if (L < m || L > 4096 || (L & (L - 1)))
    return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: pad_len %d invalid for %d channels", L, m);
  if (!(pp.ratio_floor > 0.f)) return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: ratio_floor must be > 0");
  if (pp.pec && (!(pp.als_p > 0.0 && pp.als_p < 1.0) || pp.als_iters < 1 || pp.als_iters > 1000))
    return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: bad ALS parameters");
  int sec = 0, window = 3, order = 0;
  double gi[9] = {};
  if (pp.sec) {
    if (pp.sec_mode == FKK_SEC_MEAN) {
      sec = 2;
    } else if (pp.sec_mode == FKK_SEC_SAVGOL) {
      sec = 1;
      window = pp.sg_window;
      if (!window) {
        window = m / 2;
        if (window % 2 == 0) --window;
        if (window < 3) window = 3;
      }
      order = pp.sg_order;
      if (window % 2 == 0 || window > m || window <= order || order < 0 || order > 2)
        return fail(ctx, FKK_ERR_INVALID_ARG,
                    "conventional_per_spectrum: Savitzky-Golay window %d / order %d (orders 0-2 supported)", window,
                    order);
      if (!window_moment_inverse(window, order, gi))
        return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: singular Savitzky-Golay moments");
    } else {
      return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: bad sec_mode");
    }
  }
  if (pp.denoise_k > 0 && (pp.denoise_k > 80 || pp.denoise_k > m || pp.denoise_k > n_spectra))
    return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: denoise_k %d exceeds min(80, M, N)", pp.denoise_k);
  if (pp.denoise_k < 0 && (pp.k_max < 1 || pp.k_max > 80 || pp.k_max > n_spectra || !(pp.rank_eps >= 0.0)))
    return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: rank rule needs 1 <= k_max <= min(80, N), rank_eps >= 0");
  if (n_spectra == 0) return FKK_OK;
  if (!i_cars || !i_ref || !im_out) return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: null pointer");
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  if (pp.denoise_k) {
    float* xk = nullptr;
    FKK_TRY(svd_denoise(ctx, i_cars, n_spectra, m, ld, pp, &xk, st));
    i_cars = xk;
    ld = m;
  }
  const double lam = pp.als_lambda > 0.0 ? pp.als_lambda : 1e4 * std::pow(m / 1000.0, 4);

  // finish-kernel launch shape (as the KK kernel: one FFT per tpf threads)
  int tpf = L / 8;
  if (tpf > kFinThreads) tpf = kFinThreads;
  if (tpf < 32) tpf = 32;
  const int nfft = kFinThreads / tpf;
  const size_t fsmem = finish_smem_bytes(L, m, nfft);
  if (fsmem > 227 * 1024)
    return fail(ctx, FKK_ERR_INVALID_ARG, "conventional_per_spectrum: %d channels need %zu B of shared memory", m, fsmem);
  FKK_CUDA(ctx, cudaFuncSetAttribute(conv_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
  int per_sm = 0;
  FKK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_finish_kernel, kFinThreads, fsmem));
  if (per_sm < 1) per_sm = 1;

  // chunk of spectra: enough threads for every SM, within the budget
  const int nblk = (m + 31) / 32;
  const size_t per_spec = (size_t)m * 4 * 2 + (pp.pec ? (size_t)m * 6 * 4 + (size_t)nblk * 4 : 0);
  int64_t chunk = std::min<int64_t>((n_spectra + 31) / 32 * 32, (int64_t)ctx->sm_count * 1024);
  float* phi = nullptr;
  fkk_status s = FKK_OK;
  for (;;) {
    phi = (float*)workspace(ctx, "conv_ws", (size_t)chunk * per_spec, &s);
    if (phi || s != FKK_ERR_BUDGET || chunk <= 32) break;
    chunk = std::max<int64_t>(32, chunk / 2 / 32 * 32);
    ctx->last_error.clear();
  }
  if (!phi) return s;
  float* sgk = nullptr;
  if (sec == 1) {
    sgk = (float*)workspace(ctx, "conv_sgk", (size_t)L * sizeof(float), &s);
    if (!sgk) return s;
    FKK_COUNT_LAUNCH(); sg_kernel_dft_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, window / 2, gi[0], gi[1], gi[2], sgk);
    FKK_CUDA(ctx, cudaGetLastError());
  }
  float* perr = phi + (size_t)chunk * m;
  float2* fac = reinterpret_cast<float2*>(perr + (size_t)chunk * m);
  unsigned* bits = reinterpret_cast<unsigned*>(fac + (size_t)chunk * m * 3);

  for (int64_t c0 = 0; c0 < n_spectra; c0 += chunk) {
    const int64_t cn = std::min<int64_t>(chunk, n_spectra - c0);
    const float* src = i_cars + c0 * ld;
    FKK_TRY(launch_kk_phase(ctx, src, cn, m, ld, i_ref, L, pp.ratio_floor, phi, m, st));
    if (pp.pec) {
      AlsArgs aa{phi, perr, fac, bits, cn, chunk, m, lam, pp.als_p, pp.als_iters};
      const unsigned grid = (unsigned)((cn + kAlsThreads - 1) / kAlsThreads);
      FKK_COUNT_LAUNCH(); als_kernel<<<grid, kAlsThreads, 0, st>>>(aa);
      FKK_CUDA(ctx, cudaGetLastError());
    }
    FinArgs fa{};
    fa.i_cars = src;
    fa.ld = ld;
    fa.i_ref = i_ref;
    fa.phi = phi;
    fa.perr = pp.pec ? perr : nullptr;
    fa.sgk = sgk;
    fa.n = cn;
    fa.m = m;
    fa.L = L;
    fa.floor_ = pp.ratio_floor;
    fa.sec = sec;
    fa.window = window;
    for (int q = 0; q < 9; ++q) fa.gi[q] = (float)gi[q];
    fa.im = im_out + c0 * ld_out;
    fa.re = re_out ? re_out + c0 * ld_out : nullptr;
    fa.ld_out = ld_out;
    const int64_t npairs = (cn + 1) / 2;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((npairs + nfft - 1) / nfft, (int64_t)ctx->sm_count * per_sm));
    FKK_COUNT_LAUNCH(); conv_finish_kernel<<<(unsigned)grid, kFinThreads, fsmem, st>>>(fa, tpf);
    FKK_CUDA(ctx, cudaGetLastError());
  }
  return FKK_OK;
}
