// Conventional per-spectrum KK on the GPU (Eq. KCARS with the surrogate
// reference of Eq. K): for each spectrum a = 1/2 ln(I/I_ref), phi = H{a}
// by a padded FFT, Im{K} = e^a sin(phi), Re{K} = e^a cos(phi).
//
// Two real spectra share one complex FFT: z = a0 + i a1.  The Hilbert
// multiplier -i sgn(m) is linear and maps the transform of each real input
// to that of its (real) Hilbert transform, so the inverse FFT of
// -i sgn(m) Z(m) is H{a0} + i H{a1}; no unpacking of the two spectra is
// needed.  A block keeps its twiddle table in shared memory and walks
// spectrum pairs in a grid-stride loop.  The same kernel, in its phase mode,
// writes phi = H{a} itself for the conventional workflow's PEC.
#include "fft.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr int kThreads = 256;

struct KKArgs {
  const float* i_cars;
  int64_t n;
  int m;
  int64_t ld;
  const float* i_ref;
  int L;
  float floor_;
  float* im;
  float* re;
  int64_t ld_out;
  long long* status;
};

// kPhase: write phi = H{a} to p.im (row stride p.ld_out) instead of Im/Re K.
template <bool kPhase>
__global__ void __launch_bounds__(kThreads) kk_pairs_kernel(KKArgs p, int tpf) {
  extern __shared__ float4 smem_raw[];
  const int L = p.L, M = p.m;
  const int nfft = blockDim.x / tpf;           // FFTs in flight per block
  const int f = threadIdx.x / tpf;             // my FFT slot
  const int t0 = threadIdx.x % tpf;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* slot = tw + L + f * (2 * L);
  float2* buf0 = slot;
  float2* buf1 = slot + L;
  float* a_base = reinterpret_cast<float*>(tw + L + nfft * 2 * L);
  float* a0 = a_base + f * (2 * M);
  float* a1 = a0 + M;
  const int left = (L - M) / 2;
  const float invL = 1.0f / (float)L;

  fill_twiddles(tw, L);
  int clamped = 0;
  const int64_t npairs = (p.n + 1) / 2;
  for (int64_t base = (int64_t)blockIdx.x * nfft; base < npairs; base += (int64_t)gridDim.x * nfft) {
    __syncthreads();  // previous iteration's outputs read; twiddles ready
    const int64_t pr = base + f;
    const bool live = pr < npairs;
    const int64_t n0 = 2 * pr, n1 = 2 * pr + 1;
    const bool has1 = live && n1 < p.n;
    // log ratio of both spectra
    for (int j = t0; j < M; j += tpf) {
      const float r = 1.0f / p.i_ref[j];
      float v0 = 0.f, v1 = 0.f;
      if (live) {
        float x = p.i_cars[n0 * p.ld + j] * r;
        if (!(x >= p.floor_)) { x = p.floor_; ++clamped; }
        v0 = 0.34657359027997264f * __log2f(x);  // (ln 2 / 2) log2
      }
      if (has1) {
        float x = p.i_cars[n1 * p.ld + j] * r;
        if (!(x >= p.floor_)) { x = p.floor_; ++clamped; }
        v1 = 0.34657359027997264f * __log2f(x);
      }
      a0[j] = v0;
      a1[j] = v1;
    }
    __syncthreads();
    // edge-replicated, centred padding into the complex buffer
    for (int t = t0; t < L; t += tpf) {
      int s = min(max(t - left, 0), M - 1);
      buf0[t] = make_float2(a0[s], a1[s]);
    }
    __syncthreads();
    int cur = fft_block<-1>(buf0, buf1, L, tw, t0, tpf);
    float2* X = cur ? buf1 : buf0;
    float2* Y = cur ? buf0 : buf1;
    for (int t = t0; t < L; t += tpf) X[t] = hilbert_mult(X[t], t, L);
    __syncthreads();
    int cur2 = fft_block<+1>(X, Y, L, tw, t0, tpf);
    float2* H = cur2 ? Y : X;
    if (live && kPhase) {
      for (int j = t0; j < M; j += tpf) {
        const float2 h = H[left + j];
        p.im[n0 * p.ld_out + j] = h.x * invL;
        if (has1) p.im[n1 * p.ld_out + j] = h.y * invL;
      }
    } else if (live) {
      for (int j = t0; j < M; j += tpf) {
        // the same operations as the register-FFT kernel (bit-identical outputs)
        const float2 h = H[left + j];
        const float ph0 = h.x * invL, ph1 = h.y * invL;
        const float e0 = exp2f(1.4426950408889634f * a0[j]);
        p.im[n0 * p.ld_out + j] = e0 * __sinf(ph0);
        if (p.re) p.re[n0 * p.ld_out + j] = e0 * __cosf(ph0);
        if (has1) {
          const float e1 = exp2f(1.4426950408889634f * a1[j]);
          p.im[n1 * p.ld_out + j] = e1 * __sinf(ph1);
          if (p.re) p.re[n1 * p.ld_out + j] = e1 * __cosf(ph1);
        }
      }
    }
  }
  // one atomic per warp for the clamp counter
  for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
  if ((threadIdx.x & 31) == 0 && clamped) atomicAdd(reinterpret_cast<unsigned long long*>(p.status + 1), (unsigned long long)clamped);
}

}  // namespace

// Shared-memory bytes for a block running nfft transforms of length L over
// M channels.
static size_t kk_smem_bytes(int L, int M, int nfft) {
  return sizeof(float2) * (size_t)L + (size_t)nfft * (2 * L * sizeof(float2) + 2 * M * sizeof(float));
}

template <bool kPhase>
static fkk_status launch_kk_impl(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                                 const float* i_ref, int L, float floor_, float* im, float* re,
                                 int64_t ld_out, cudaStream_t st) {
  bool handled = false;
  fkk_status ws = launch_kk_warp(ctx, i_cars, n, m, ld, i_ref, L, floor_, im, re, ld_out, kPhase, st, &handled);
  if (handled) return ws;
  int tpf = L / 8;
  if (tpf > kThreads) tpf = kThreads;
  if (tpf < 32) tpf = 32;
  int nfft = kThreads / tpf;
  size_t smem = kk_smem_bytes(L, m, nfft);
  if (smem > 227 * 1024) return fail(ctx, FKK_ERR_INVALID_ARG, "pad_len %d with %d channels needs %zu B of shared memory", L, m, smem);
  FKK_CUDA(ctx, cudaFuncSetAttribute(kk_pairs_kernel<kPhase>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FKK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kk_pairs_kernel<kPhase>, kThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t npairs = (n + 1) / 2;
  int64_t want = (npairs + nfft - 1) / nfft;
  int64_t grid = std::min<int64_t>(want, (int64_t)ctx->sm_count * per_sm);
  if (grid < 1) grid = 1;
  KKArgs a{i_cars, n, m, ld, i_ref, L, floor_, im, re, ld_out, ctx->d_status};
  FKK_COUNT_LAUNCH(); kk_pairs_kernel<kPhase><<<(unsigned)grid, kThreads, smem, st>>>(a, tpf);
  return cuda_check(ctx, cudaGetLastError(), "kk_pairs_kernel launch");
}

fkk_status launch_kk(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                     const float* i_ref, int L, float floor_, float* im, float* re,
                     int64_t ld_out, cudaStream_t st) {
  return launch_kk_impl<false>(ctx, i_cars, n, m, ld, i_ref, L, floor_, im, re, ld_out, st);
}

fkk_status launch_kk_phase(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                           const float* i_ref, int L, float floor_, float* phi, int64_t ld_phi,
                           cudaStream_t st) {
  return launch_kk_impl<true>(ctx, i_cars, n, m, ld, i_ref, L, floor_, phi, nullptr, ld_phi, st);
}

}  // namespace fkk

using namespace fkk;

extern "C" fkk_status kk_per_spectrum(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra,
                                      int32_t n_channels, int64_t ld, const float* i_ref,
                                      int32_t pad_len, float ratio_floor, float* im_out,
                                      float* re_out, int64_t ld_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (n_spectra < 0 || n_channels < 1 || ld < n_channels || ld_out < n_channels)
    return fail(ctx, FKK_ERR_INVALID_ARG, "kk_per_spectrum: bad sizes (n=%lld m=%d ld=%lld ld_out=%lld)",
                (long long)n_spectra, n_channels, (long long)ld, (long long)ld_out);
  if (!(ratio_floor > 0.f)) return fail(ctx, FKK_ERR_INVALID_ARG, "kk_per_spectrum: ratio_floor must be > 0");
  int L = pad_len ? pad_len : next_pow2(2 * (int64_t)n_channels);
  if (L < n_channels || L > 8192 || L < 2 || (L & (L - 1)))
    return fail(ctx, FKK_ERR_INVALID_ARG, "kk_per_spectrum: pad_len %d invalid for %d channels", L, n_channels);
  if (n_spectra == 0) return FKK_OK;
  if (!i_cars || !i_ref || !im_out) return fail(ctx, FKK_ERR_INVALID_ARG, "kk_per_spectrum: null pointer");
  FKK_TRY(bind(ctx));
  return launch_kk(ctx, i_cars, n_spectra, n_channels, ld, i_ref, L, ratio_floor, im_out, re_out, ld_out,
                   as_stream(stream));
}
