// C-ABI entry points of the fKK-EC fit, the ML apply, the basis object and
// the individual pipeline steps (include/fkk.h).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "fit.h"

#include "basis_internal.h"

namespace fkk {
namespace {

__global__ void f_from_f32_kernel(const float* __restrict__ src, int m, double* __restrict__ f) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) f[j] = src ? (double)src[j] : 1.0;
}

__global__ void s_and_w_kernel(const double* __restrict__ lam, const double* __restrict__ v, int m, int k,
                               double ml_lambda, double* __restrict__ s, double* __restrict__ w) {
  const int i = blockIdx.x;
  const double l = lam[i] > 0.0 ? lam[i] : 0.0;
  const double shrink = (l + ml_lambda) > 0.0 ? l / (l + ml_lambda) : 0.0;
  if (threadIdx.x == 0) s[i] = sqrt(l);
  for (int j = threadIdx.x; j < m; j += blockDim.x) w[(int64_t)j * k + i] = v[(int64_t)j * k + i] * shrink;
}

// Training mean of the log ratios per channel, 1/2 ln max(I/I_ref, floor):
// the transform's shift c plus the mean of the shifted values.
__global__ void offset_kernel(const float* __restrict__ c, const double* __restrict__ sum_d, int64_t n, int m,
                              double* __restrict__ a_off) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) a_off[j] = (double)c[j] + sum_d[j] / (double)n;
}

__global__ void copy_f32_kernel(const float* __restrict__ a, int m, float* __restrict__ b) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) b[j] = a[j];
}

// *out = ||A||_F^2 = sum_j f_j^2 (sum_n d^2 + 2 c_j sum_n d + n c_j^2) (d the
// shifted log ratio, a = d + c), one block.
__global__ void energy_kernel(const double* __restrict__ sd2, const double* __restrict__ sd,
                              const float* __restrict__ c, const double* __restrict__ f, int64_t n, int m,
                              double* __restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double cj = c[j];
    t += f[j] * f[j] * (sd2[j] + 2.0 * cj * sd[j] + (double)n * cj * cj);
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
    *out = u;
  }
}

// *out = trace(G), one block.
__global__ void trace_kernel(const double* __restrict__ g, int m, double* __restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) t += g[(int64_t)j * m + j];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
    *out = u;
  }
}

// acc[0] += sum over rows of ||f a||^2 (a = 1/2 ln max(I/I_ref, floor)),
// acc[1] += sum of P^2 (n x k).  A warp per row, fp64 block sums.
__global__ void residual_energy_kernel(const float* __restrict__ i_cars, int64_t n, int m, int64_t ld,
                                       const float* __restrict__ i_ref, float floor_, const double* __restrict__ f,
                                       const float* __restrict__ p, int k, double* __restrict__ acc) {
  __shared__ double red[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double ea = 0.0, ep = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * nw + warp; r < n; r += (int64_t)gridDim.x * nw) {
    float sa = 0.f;
    for (int j = lane; j < m; j += 32) {
      float x = i_cars[r * ld + j] / i_ref[j];
      if (!(x >= floor_)) x = floor_;
      const float a = (float)f[j] * 0.5f * logf(x);
      sa = fmaf(a, a, sa);
    }
    float sp = 0.f;
    for (int i = lane; i < k; i += 32) {
      const float v = p[r * k + i];
      sp = fmaf(v, v, sp);
    }
    ea += sa;
    ep += sp;
  }
  ea = warp_sum(ea);
  ep = warp_sum(ep);
  if (lane == 0) {
    red[0][warp] = ea;
    red[1][warp] = ep;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, v = 0.0;
    for (int w = 0; w < nw; ++w) {
      u += red[0][w];
      v += red[1][w];
    }
    atomicAdd(acc, u);
    atomicAdd(acc + 1, v);
  }
}

fkk_status check_params(fkk_ctx* ctx, const fkk_fit_params& p, int m, int64_t n) {
  if (p.k == 0) {
    if (p.k_max < 1 || p.k_max > 80) return fail(ctx, FKK_ERR_INVALID_ARG, "k_max=%d must be in [1, 80]", p.k_max);
    if (!(p.rank_eps >= 0.0)) return fail(ctx, FKK_ERR_INVALID_ARG, "rank_eps must be >= 0");
  } else {
    if (p.k < 1 || p.k > 80 || p.k > m) return fail(ctx, FKK_ERR_INVALID_ARG, "k=%d must be in [1, min(80, M)]", p.k);
    if (n < p.k) return fail(ctx, FKK_ERR_INVALID_ARG, "need at least k spectra");
  }
  if (p.pad_len && (p.pad_len < m || p.pad_len > 4096 || (p.pad_len & (p.pad_len - 1))))
    return fail(ctx, FKK_ERR_INVALID_ARG, "pad_len %d invalid", p.pad_len);
  if (!p.pad_len && next_pow2(2 * (int64_t)m) > 4096)
    return fail(ctx, FKK_ERR_INVALID_ARG, "n_channels %d too large for the basis Hilbert transform", m);
  if (!(p.als_p > 0.0 && p.als_p < 1.0) || p.als_iters < 1) return fail(ctx, FKK_ERR_INVALID_ARG, "bad ALS parameters");
  if (!(p.ridge_rel >= 0.0) || !(p.ml_lambda >= 0.0)) return fail(ctx, FKK_ERR_INVALID_ARG, "negative ridge");
  if (p.sec_mode != FKK_SEC_SAVGOL && p.sec_mode != FKK_SEC_MEAN) return fail(ctx, FKK_ERR_INVALID_ARG, "bad sec_mode");
  if (p.sec && p.sec_mode == FKK_SEC_SAVGOL) {
    int w = p.sg_window;
    if (w && (w % 2 == 0 || w > m || w <= p.sg_order)) return fail(ctx, FKK_ERR_INVALID_ARG, "bad sg_window");
    if (p.sg_order < 0 || p.sg_order > 7) return fail(ctx, FKK_ERR_INVALID_ARG, "bad sg_order");
  }
  if (!(p.ratio_floor > 0.f)) return fail(ctx, FKK_ERR_INVALID_ARG, "ratio_floor must be > 0");
  if (p.precision != FKK_PREC_BF16X3 && p.precision != FKK_PREC_BF16)
    return fail(ctx, FKK_ERR_INVALID_ARG, "unknown precision %d", p.precision);
  if (p.noise_alpha < 0.0 || p.noise_sigma_g < 0.0) return fail(ctx, FKK_ERR_INVALID_ARG, "negative noise parameter");
  if (p.svd != FKK_SVD_EXACT && p.svd != FKK_SVD_RANDOMIZED) return fail(ctx, FKK_ERR_INVALID_ARG, "bad svd");
  if (p.svd == FKK_SVD_RANDOMIZED) {
    if (p.k < 1) return fail(ctx, FKK_ERR_INVALID_ARG, "the randomised SVD needs k >= 1");
    if (p.rsvd_oversample < 0 || p.k + p.rsvd_oversample > 80)
      return fail(ctx, FKK_ERR_INVALID_ARG, "randomised SVD: k + oversample = %d must be <= 80", p.k + p.rsvd_oversample);
    if (p.rsvd_power_iters < 0 || p.rsvd_power_iters > 20)
      return fail(ctx, FKK_ERR_INVALID_ARG, "randomised SVD: power_iters %d not in 0..20", p.rsvd_power_iters);
    if (p.refine_steps != 0)
      return fail(ctx, FKK_ERR_INVALID_ARG, "refine_steps applies to the exact SVD (the randomised SVD refines "
                                            "through rsvd_power_iters)");
  }
  if (p.refine_steps < 0 || p.refine_steps > 4)
    return fail(ctx, FKK_ERR_INVALID_ARG, "refine_steps %d not in 0..4", p.refine_steps);
  return FKK_OK;
}

BasisParams basis_params(const fkk_fit_params& p, int m, int L) {
  BasisParams bp;
  bp.m = m;
  bp.k = p.k;
  bp.L = L;
  bp.pec = p.pec;
  bp.sec = p.sec;
  bp.als_lambda = p.als_lambda > 0.0 ? p.als_lambda : 1e4 * std::pow(m / 1000.0, 4);
  bp.als_p = p.als_p;
  bp.als_iters = p.als_iters;
  bp.ridge_rel = p.ridge_rel;
  bp.sec_mode = p.sec_mode;
  int w = p.sg_window;
  if (!w) {
    w = m / 2;
    if (w % 2 == 0) --w;
    if (w < 3) w = 3;
  }
  bp.sg_window = w;
  bp.sg_order = p.sg_order;
  return bp;
}

// Bytes of the single device block backing a basis of m channels and k
// vectors (the layout basis_alloc carves up).
size_t basis_block_bytes(int m, int k) {
  const size_t mk = (size_t)m * k;
  const size_t doubles = (size_t)m + 2 * k + 2 * mk + 7 * mk + (size_t)m;  // ... c_ph, then a_off (m)
  return doubles * 8 + (size_t)2 * k * 8 + 64 + (size_t)m * 4 + 256;
}

fkk_basis* basis_alloc(fkk_ctx* ctx, int m, int k, fkk_status* st) {
  fkk_basis* b = new (std::nothrow) fkk_basis();
  if (!b) {
    *st = FKK_ERR_INVALID_ARG;
    return nullptr;
  }
  const size_t mk = (size_t)m * k;
  cudaError_t e = cudaMalloc(&b->block, basis_block_bytes(m, k));
  if (e != cudaSuccess) {
    *st = cuda_check(ctx, e, "cudaMalloc(basis)");
    delete b;
    return nullptr;
  }
  double* d = (double*)b->block;
  b->f = d; d += m;
  b->lam = d; d += k;
  b->s = d; d += k;
  b->v = d; d += mk;
  b->w = d; d += mk;
  b->b = d; d += mk;
  b->h_b = d; d += mk;
  b->phi_pec_t = d; d += mk;
  b->h_phi = d; d += mk;
  b->v_sec_t = d; d += mk;
  b->c_amp = d; d += mk;
  b->c_ph = d; d += mk;
  b->a_off = d; d += m;
  b->q = (int64_t*)d;
  b->nq = (int*)(b->q + 2 * k);
  b->energy = reinterpret_cast<double*>(b->nq) + 1;
  b->i_ref = (float*)(reinterpret_cast<uint8_t*>(b->nq) + 64);
  b->device = ctx->device;
  b->m = m;
  b->k = k;
  *st = FKK_OK;
  return b;
}

}  // namespace
}  // namespace fkk

using namespace fkk;

extern "C" {

void fkk_fit_params_default(fkk_fit_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->k = 20;
  p->pad_len = 0;
  p->pec = 1;
  p->sec = 1;
  p->als_lambda = 0.0;
  p->als_p = 0.01;
  p->als_iters = 20;
  p->ridge_rel = 1e-3;
  p->sec_mode = FKK_SEC_SAVGOL;
  p->sg_window = 0;
  p->sg_order = 2;
  p->ml_lambda = 0.0;
  p->precision = FKK_PREC_BF16X3;
  p->ratio_floor = 1e-6f;
  p->noise_alpha = 0.0;
  p->noise_sigma_g = 0.0;
  p->k_max = 80;
  p->rank_eps = 0.0;
  p->refine_steps = 0;
  p->svd = FKK_SVD_EXACT;
  p->rsvd_oversample = 10;
  p->rsvd_power_iters = 2;
  p->rsvd_seed = 0;
  p->denoise_k = 0;
}

fkk_status fkk_fit_basis(fkk_ctx* ctx, const float* i_cars, int64_t n, int32_t m, int64_t ld, const float* i_ref,
                         const float* f_or_null, const fkk_fit_params* params, fkk_basis** out_basis,
                         float* im_out, float* re_out, int64_t ld_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!params || !out_basis || !i_cars || !i_ref) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_fit_basis: null argument");
  if (m < 8 || m > 2048 || n < 1 || ld < m) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_fit_basis: bad sizes");
  if ((im_out || re_out) && ld_out < m) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_fit_basis: bad ld_out");
  FKK_TRY(check_params(ctx, *params, m, n));
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  // Host buffers (pinned or pageable) are staged through the context's
  // workspace on `stream`: inputs copied in before the transform, outputs
  // copied back after the reconstruction.  Device pointers are used in place.
  const bool im_on_host = im_out && is_host_ptr(im_out), re_on_host = re_out && is_host_ptr(re_out);
  if ((im_out && re_out) && im_on_host != re_on_host)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_fit_basis: im_out and re_out must both be host or both device memory");
  float* im_host = nullptr;
  float* re_host = nullptr;
  const int64_t ld_host = ld_out;
  {
    fkk_status sh;
    if (is_host_ptr(i_cars)) {
      float* d = (float*)workspace(ctx, "fit_host_x", (size_t)n * m * 4, &sh);
      if (!d) return sh;
      if (ld == m)  // packed rows: one linear copy (a pitched copy moves row by row)
        FKK_CUDA(ctx, cudaMemcpyAsync(d, i_cars, (size_t)n * m * 4, cudaMemcpyHostToDevice, st));
      else
        FKK_CUDA(ctx, cudaMemcpy2DAsync(d, (size_t)m * 4, i_cars, (size_t)ld * 4, (size_t)m * 4, (size_t)n,
                                        cudaMemcpyHostToDevice, st));
      i_cars = d;
      ld = m;
    }
    if (is_host_ptr(i_ref)) {
      float* d = (float*)workspace(ctx, "fit_host_ref", (size_t)m * 4, &sh);
      if (!d) return sh;
      FKK_CUDA(ctx, cudaMemcpyAsync(d, i_ref, (size_t)m * 4, cudaMemcpyHostToDevice, st));
      i_ref = d;
    }
    if (f_or_null && is_host_ptr(f_or_null)) {
      float* d = (float*)workspace(ctx, "fit_host_f", (size_t)m * 4, &sh);
      if (!d) return sh;
      FKK_CUDA(ctx, cudaMemcpyAsync(d, f_or_null, (size_t)m * 4, cudaMemcpyHostToDevice, st));
      f_or_null = d;
    }
    if (im_on_host || re_on_host) {
      if (im_out) {
        im_host = im_out;
        im_out = (float*)workspace(ctx, "fit_host_im", (size_t)n * m * 4, &sh);
        if (!im_out) return sh;
      }
      if (re_out) {
        re_host = re_out;
        re_out = (float*)workspace(ctx, "fit_host_re", (size_t)n * m * 4, &sh);
        if (!re_out) return sh;
      }
      ld_out = m;
    }
  }
  fkk_fit_params p = *params;  // k is filled in below when chosen by the rank rule
  const bool autok = p.k == 0;
  int k = p.k;
  const int L = p.pad_len ? p.pad_len : next_pow2(2 * (int64_t)m);
  fkk_status s;
  fkk_basis* B = nullptr;
  auto bail = [&](fkk_status e) {
    cudaStreamSynchronize(st);
    if (B) {
      cudaFree(B->block);
      delete B;
    }
    return e;
  };
  double* f_dev = nullptr;  // f(w): the basis' own array, or a workspace until k is known
  if (autok) {
    f_dev = (double*)workspace(ctx, "fit_f_auto", (size_t)m * 8, &s);
    if (!f_dev) return s;
  } else {
    B = basis_alloc(ctx, m, k, &s);
    if (!B) return s;
    f_dev = B->f;
  }
  DtLayout D;
  stage_mark(ctx, 0, st);
  s = launch_transform(ctx, i_cars, n, m, ld, i_ref, p.ratio_floor, D, st);
  if (s) return bail(s);
  // f(w)
  if (f_or_null) {
    FKK_COUNT_LAUNCH(); f_from_f32_kernel<<<(m + 127) / 128, 128, 0, st>>>(f_or_null, m, f_dev);
  } else if (p.noise_alpha > 0.0 || p.noise_sigma_g > 0.0) {
    s = launch_noise_scale(ctx, D.sum_i, n, m, p.noise_alpha, p.noise_sigma_g, f_dev, st);
    if (s) return bail(s);
  } else {
    FKK_COUNT_LAUNCH(); f_from_f32_kernel<<<(m + 127) / 128, 128, 0, st>>>(nullptr, m, f_dev);
  }
  double* G = nullptr;
  stage_mark(ctx, 1, st);
  if (p.svd == FKK_SVD_RANDOMIZED) {  // k fixed: B was allocated above, f_dev is B->f
    stage_mark(ctx, 2, st);
    if ((s = launch_rsvd(ctx, D, B->f, k, p.rsvd_oversample, p.rsvd_power_iters, p.rsvd_seed, B->lam, B->v, st)))
      return bail(s);
  } else {
    G = (double*)workspace(ctx, "fit_gram", (size_t)m * m * 8, &s);
    if (!G) return bail(s);
    if ((s = launch_gram(ctx, D, f_dev, G, st))) return bail(s);
    stage_mark(ctx, 2, st);
    if (autok) {
      // the k_max largest eigenpairs, then the rank rule on the host
      const int kmax = std::min(p.k_max, m);
      double* lam_a = (double*)workspace(ctx, "fit_lam_auto", (size_t)kmax * 8, &s);
      if (!lam_a) return bail(s);
      double* v_a = (double*)workspace(ctx, "fit_v_auto", (size_t)m * kmax * 8, &s);
      if (!v_a) return bail(s);
      if ((s = launch_eig_topk(ctx, G, m, kmax, lam_a, v_a, st))) return bail(s);
      std::vector<double> lam(kmax);
      if ((s = cuda_check(ctx, cudaMemcpyAsync(lam.data(), lam_a, kmax * 8, cudaMemcpyDeviceToHost, st), "lambda")))
        return bail(s);
      if ((s = cuda_check(ctx, cudaStreamSynchronize(st), "rank rule"))) return bail(s);
      const double eps = p.rank_eps > 0.0 ? p.rank_eps : (double)FLT_EPSILON;
      const double tol = std::sqrt(std::max(lam[0], 0.0)) * (double)std::max<int64_t>(n, m) * eps;
      k = 0;
      while (k < kmax && std::sqrt(std::max(lam[k], 0.0)) > tol) ++k;
      if (k < 1) k = 1;
      p.k = k;
      B = basis_alloc(ctx, m, k, &s);
      if (!B) return bail(s);
      if ((s = cuda_check(ctx, cudaMemcpyAsync(B->f, f_dev, (size_t)m * 8, cudaMemcpyDeviceToDevice, st), "f")) ||
          (s = cuda_check(ctx, cudaMemcpyAsync(B->lam, lam_a, (size_t)k * 8, cudaMemcpyDeviceToDevice, st), "lambda")) ||
          (s = cuda_check(ctx, cudaMemcpy2DAsync(B->v, (size_t)k * 8, v_a, (size_t)kmax * 8, (size_t)k * 8, m,
                                                 cudaMemcpyDeviceToDevice, st), "V")))
        return bail(s);
    } else {
      if ((s = launch_eig_topk(ctx, G, m, k, B->lam, B->v, st))) return bail(s);
    }
    if (p.refine_steps > 0 && (s = launch_refine(ctx, G, m, k, B->v, p.refine_steps, B->lam, B->v, st)))
      return bail(s);
  }
  B->params = p;
  B->L = L;
  FKK_COUNT_LAUNCH(); copy_f32_kernel<<<(m + 127) / 128, 128, 0, st>>>(i_ref, m, B->i_ref);
  if (G) {
    FKK_COUNT_LAUNCH(); trace_kernel<<<1, 256, 0, st>>>(G, m, B->energy);
  } else {
    FKK_COUNT_LAUNCH(); energy_kernel<<<1, 256, 0, st>>>(D.sum_d2, D.sum_d, D.c, B->f, n, m, B->energy);
  }
  FKK_COUNT_LAUNCH(); s_and_w_kernel<<<k, 256, 0, st>>>(B->lam, B->v, m, k, p.ml_lambda, B->s, B->w);
  FKK_COUNT_LAUNCH(); offset_kernel<<<(m + 127) / 128, 128, 0, st>>>(D.c, D.sum_d, n, m, B->a_off);
  float* P = (float*)workspace(ctx, "fit_p", (size_t)n * k * 4, &s);
  if (!P) return bail(s);
  int64_t* qm = (int64_t*)workspace(ctx, "fit_qext", (size_t)2 * k * 8, &s);
  if (!qm) return bail(s);
  stage_mark(ctx, 3, st);
  if ((s = launch_project(ctx, D, B->v, B->f, k, P, qm, qm + k, st))) return bail(s);
  stage_mark(ctx, 4, st);
  int* nq_dev = (int*)workspace(ctx, "fit_nq", 64, &s);
  if (!nq_dev) return bail(s);
  double* xr = (double*)workspace(ctx, "fit_xrows", (size_t)2 * k * k * 8, &s);
  if (!xr) return bail(s);
  if ((s = launch_gather_q(ctx, qm, qm + k, k, P, n, B->q, nq_dev, xr, st))) return bail(s);
  if ((s = cuda_check(ctx, cudaMemcpyAsync(B->nq, nq_dev, sizeof(int), cudaMemcpyDeviceToDevice, st), "nq"))) return bail(s);
  BasisOut bo{B->c_amp, B->c_ph, B->b, B->h_b, B->phi_pec_t, B->h_phi, B->v_sec_t};
  if ((s = launch_basis_math(ctx, basis_params(p, m, L), B->v, B->f, xr, 2 * k, bo, st))) return bail(s);
  stage_mark(ctx, 5, st);
  if (im_out) {
    if ((s = launch_reconstruct(ctx, P, n, k, m, B->c_amp, B->c_ph, im_out, re_out, ld_out, st))) return bail(s);
    // device-to-host: one linear copy when the host rows are packed
    auto to_host = [&](float* dst, const float* src, const char* what) {
      if (ld_host == m)
        return cuda_check(ctx, cudaMemcpyAsync(dst, src, (size_t)n * m * 4, cudaMemcpyDeviceToHost, st), what);
      return cuda_check(ctx, cudaMemcpy2DAsync(dst, (size_t)ld_host * 4, src, (size_t)m * 4, (size_t)m * 4, (size_t)n,
                                               cudaMemcpyDeviceToHost, st), what);
    };
    if (im_host && (s = to_host(im_host, im_out, "copy Im to host"))) return bail(s);
    if (re_host && (s = to_host(re_host, re_out, "copy Re to host"))) return bail(s);
  }
  stage_mark(ctx, 6, st);
  if ((s = cuda_check(ctx, cudaGetLastError(), "fkk_fit_basis"))) return bail(s);
  *out_basis = B;
  return FKK_OK;
}

fkk_status fkk_apply(fkk_ctx* ctx, const fkk_basis* B, const float* i_cars, int64_t n, int64_t ld, float* im_out,
                     float* re_out, int64_t ld_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!B) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_apply: null basis");
  if (n < 0 || ld < B->m || ld_out < B->m) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_apply: bad sizes");
  if (n == 0) return FKK_OK;
  if (!i_cars || !im_out) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_apply: null array");
  if (B->device != ctx->device) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_apply: basis on another device");
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  fkk_status s;
  bool handled = false;
  FKK_TRY(launch_apply_fused(ctx, B, i_cars, n, ld, im_out, re_out, ld_out, st, &handled));
  if (handled) return FKK_OK;
  // strides or alignments TMA cannot address, or k > 62: the fit's
  // transform (log ratios as bf16 hi / lo, channel-major), its tensor-core
  // projection and the reconstruction (fp32-accurate in either precision)
  float* P = (float*)workspace(ctx, "apply_p", (size_t)n * B->k * 4, &s);
  if (!P) return s;
  DtLayout D;
  FKK_TRY(launch_transform(ctx, i_cars, n, B->m, ld, B->i_ref, B->params.ratio_floor, D, st));
  FKK_TRY(launch_project(ctx, D, B->w, B->f, B->k, P, nullptr, nullptr, st));
  return launch_reconstruct(ctx, P, n, B->k, B->m, B->c_amp, B->c_ph, im_out, re_out, ld_out, st);
}

fkk_status fkk_residual(fkk_ctx* ctx, const fkk_basis* B, const float* i_cars, int64_t n, int64_t ld,
                        double* frac_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!B || !frac_out || !i_cars || n < 1 || ld < B->m) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_residual: bad arguments");
  if (B->device != ctx->device) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_residual: basis on another device");
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  fkk_status s;
  float* P = (float*)workspace(ctx, "resid_p", (size_t)n * B->k * 4, &s);
  if (!P) return s;
  double* acc = (double*)workspace(ctx, "resid_acc", 16, &s);
  if (!acc) return s;
  FKK_CUDA(ctx, cudaMemsetAsync(acc, 0, 16, st));
  // P = A V (the orthonormal V, not the apply's shrunk W)
  FKK_TRY(launch_project_raw(ctx, i_cars, n, B->m, ld, B->i_ref, B->params.ratio_floor, B->v, B->f, B->k, P, st));
  const int grid = (int)std::min<int64_t>((n + 7) / 8, (int64_t)ctx->sm_count * 8);
  FKK_COUNT_LAUNCH();
  residual_energy_kernel<<<grid, 256, 0, st>>>(i_cars, n, B->m, ld, B->i_ref, B->params.ratio_floor, B->f, P, B->k, acc);
  FKK_CUDA(ctx, cudaGetLastError());
  double h[2];
  FKK_CUDA(ctx, cudaMemcpyAsync(h, acc, 16, cudaMemcpyDeviceToHost, st));
  FKK_CUDA(ctx, cudaStreamSynchronize(st));
  *frac_out = h[0] > 0.0 ? 1.0 - h[1] / h[0] : 0.0;
  return FKK_OK;
}

size_t fkk_fit_params_size(void) { return sizeof(fkk_fit_params); }

fkk_status fkk_basis_from_arrays(fkk_ctx* ctx, int32_t m, const fkk_fit_params* params, const double* f,
                                 const double* sv, const double* v, const double* c_amp, const double* c_ph,
                                 const double* i_ref, fkk_basis** out) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!params || !f || !sv || !v || !c_amp || !c_ph || !i_ref || !out || m < 8 || m > 2048)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_basis_from_arrays: bad arguments");
  if (params->k < 1) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_basis_from_arrays: k must be >= 1");
  FKK_TRY(check_params(ctx, *params, m, params->k));
  FKK_TRY(bind(ctx));
  const int k = params->k;
  fkk_status s;
  fkk_basis* B = basis_alloc(ctx, m, k, &s);
  if (!B) return s;
  B->params = *params;
  B->L = params->pad_len ? params->pad_len : next_pow2(2 * (int64_t)m);
  const size_t mk = (size_t)m * k;
  std::vector<double> lam(k), w(mk);
  for (int i = 0; i < k; ++i) lam[i] = sv[i] * sv[i];
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < k; ++i) {
      const double l = lam[i];
      const double shrink = (l + params->ml_lambda) > 0.0 ? l / (l + params->ml_lambda) : 0.0;
      w[(size_t)j * k + i] = v[(size_t)j * k + i] * shrink;
    }
  std::vector<float> ir(m);
  for (int j = 0; j < m; ++j) ir[j] = (float)i_ref[j];
  int zero = 0;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cp(B->f, f, m * 8);
  cp(B->s, sv, k * 8);
  cp(B->lam, lam.data(), k * 8);
  cp(B->v, v, mk * 8);
  cp(B->w, w.data(), mk * 8);
  cp(B->c_amp, c_amp, mk * 8);
  cp(B->c_ph, c_ph, mk * 8);
  if (e == cudaSuccess) e = cudaMemset(B->a_off, 0, (size_t)m * 8);
  cp(B->i_ref, ir.data(), m * 4);
  cp(B->nq, &zero, sizeof zero);
  const double no_energy = 0.0;  // unknown for an imported basis
  cp(B->energy, &no_energy, sizeof no_energy);
  if (e == cudaSuccess) e = cudaMemset(B->b, 0, 5 * mk * 8);  // b .. v_sec_t are not part of an imported basis
  if (e != cudaSuccess) {
    s = cuda_check(ctx, e, "fkk_basis_from_arrays");
    cudaFree(B->block);
    delete B;
    return s;
  }
  B->params.pec = 0;  // no sub-sample to report
  *out = B;
  return FKK_OK;
}

// ------------------------------------------------------ save / load ---
// File: 8-byte magic, u32 format version, u32 sizeof(fkk_fit_params),
// i32 m, k, pad_len, u32 0, u64 block bytes, u64 FNV-1a of the block, the
// parameter struct, then the device block byte for byte (all arrays of the
// basis in the layout basis_alloc defines).
namespace {
constexpr char kMagic[8] = {'F', 'K', 'K', 'B', 'A', 'S', 'I', 'S'};
constexpr uint32_t kFormat = 3;  // 2: the training offset of the log ratios follows C_ph; 3: refine_steps
struct FileHead {
  char magic[8];
  uint32_t version;
  uint32_t params_size;
  int32_t m, k, L;
  uint32_t pad;
  uint64_t block_bytes;
  uint64_t checksum;
};
uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}
}  // namespace

fkk_status fkk_basis_save(const fkk_basis* b, const char* path) {
  if (!b || !path) return FKK_ERR_INVALID_ARG;
  const size_t bytes = basis_block_bytes(b->m, b->k);
  std::vector<uint8_t> host(bytes);
  if (cudaSetDevice(b->device) != cudaSuccess) return FKK_ERR_CUDA;
  if (cudaMemcpy(host.data(), b->block, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return FKK_ERR_CUDA;
  FileHead h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = kFormat;
  h.params_size = sizeof(fkk_fit_params);
  h.m = b->m;
  h.k = b->k;
  h.L = b->L;
  h.block_bytes = bytes;
  h.checksum = fnv1a(host.data(), bytes);
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return FKK_ERR_BAD_FILE;
  bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 && std::fwrite(&b->params, sizeof b->params, 1, fp) == 1 &&
            std::fwrite(host.data(), 1, bytes, fp) == bytes;
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? FKK_OK : FKK_ERR_BAD_FILE;
}

fkk_status fkk_basis_load(fkk_ctx* ctx, const char* path, fkk_basis** out) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!path || !out) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_basis_load: null argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(ctx, FKK_ERR_BAD_FILE, "fkk_basis_load: cannot open %s", path);
  FileHead h{};
  fkk_fit_params p{};
  auto bad = [&](const char* why) {
    std::fclose(fp);
    return fail(ctx, FKK_ERR_BAD_FILE, "fkk_basis_load: %s", why);
  };
  if (std::fread(&h, sizeof h, 1, fp) != 1) return bad("truncated header");
  if (std::memcmp(h.magic, kMagic, 8) != 0) return bad("not a basis file");
  if (h.version != kFormat) return bad("unsupported format version");
  if (h.params_size != sizeof(fkk_fit_params)) return bad("parameter block of another layout");
  if (h.m < 2 || h.m > 2048 || h.k < 1 || h.k > 80 || h.k > h.m) return bad("sizes out of range");
  if (h.block_bytes != basis_block_bytes(h.m, h.k)) return bad("block size does not match m and k");
  if (std::fread(&p, sizeof p, 1, fp) != 1) return bad("truncated parameters");
  std::vector<uint8_t> host(h.block_bytes);
  if (std::fread(host.data(), 1, h.block_bytes, fp) != h.block_bytes) return bad("truncated data");
  std::fclose(fp);
  if (fnv1a(host.data(), host.size()) != h.checksum) return fail(ctx, FKK_ERR_BAD_FILE, "fkk_basis_load: checksum mismatch");
  if (p.k != h.k) return fail(ctx, FKK_ERR_BAD_FILE, "fkk_basis_load: parameters disagree with the header");
  FKK_TRY(bind(ctx));
  fkk_status s;
  fkk_basis* B = basis_alloc(ctx, h.m, h.k, &s);
  if (!B) return s;
  B->params = p;
  B->L = h.L;
  const cudaError_t e = cudaMemcpy(B->block, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(B->block);
    delete B;
    return cuda_check(ctx, e, "fkk_basis_load: upload");
  }
  *out = B;
  return FKK_OK;
}

fkk_status fkk_basis_set_offset(fkk_basis* b, const double* offset, int32_t n_channels) {
  if (!b || !offset || n_channels != b->m) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->pack_mu);
  if (cudaSetDevice(b->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FKK_ERR_CUDA;
  if (cudaMemcpy(b->a_off, offset, (size_t)b->m * 8, cudaMemcpyHostToDevice) != cudaSuccess) return FKK_ERR_CUDA;
  if (b->pack) {  // the packed operands carry the offset: rebuild on next use
    cudaFree(b->pack);
    b->pack = nullptr;
  }
  return FKK_OK;
}

fkk_status fkk_basis_set_precision(fkk_basis* b, int32_t precision) {
  if (!b || (precision != FKK_PREC_BF16X3 && precision != FKK_PREC_BF16)) return FKK_ERR_INVALID_ARG;
  b->params.precision = precision;
  return FKK_OK;
}

void fkk_basis_free(fkk_basis* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  cudaFree(b->block);
  if (b->pack) cudaFree(b->pack);
  delete b;
}

fkk_status fkk_basis_info(const fkk_basis* b, int32_t* m, int32_t* k, int32_t* L, int32_t* nq) {
  if (!b) return FKK_ERR_INVALID_ARG;
  if (m) *m = b->m;
  if (k) *k = b->k;
  if (L) *L = b->L;
  if (nq) {
    if (cudaSetDevice(b->device) != cudaSuccess) return FKK_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return FKK_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, b->nq, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return FKK_ERR_CUDA;
    *nq = b->params.pec ? v : 0;
  }
  return FKK_OK;
}

fkk_status fkk_basis_get(const fkk_basis* b, int32_t which, double* dst, size_t count) {
  if (!b || !dst) return FKK_ERR_INVALID_ARG;
  const size_t mk = (size_t)b->m * b->k;
  const double* src = nullptr;
  size_t want = 0;
  switch (which) {
    case FKK_ART_S: src = b->s; want = b->k; break;
    case FKK_ART_LAMBDA: src = b->lam; want = b->k; break;
    case FKK_ART_V: src = b->v; want = mk; break;
    case FKK_ART_F: src = b->f; want = b->m; break;
    case FKK_ART_B: src = b->b; want = mk; break;
    case FKK_ART_H_B: src = b->h_b; want = mk; break;
    case FKK_ART_PHI_PEC: src = b->phi_pec_t; want = mk; break;
    case FKK_ART_H_PHI: src = b->h_phi; want = mk; break;
    case FKK_ART_V_SEC: src = b->v_sec_t; want = mk; break;
    case FKK_ART_C_AMP: src = b->c_amp; want = mk; break;
    case FKK_ART_C_PH: src = b->c_ph; want = mk; break;
    case FKK_ART_Q: break;
    case FKK_ART_ENERGY: src = b->energy; want = 1; break;
    default: return FKK_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(b->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FKK_ERR_CUDA;
  if (which == FKK_ART_Q) {
    int nq = 0;
    if (cudaMemcpy(&nq, b->nq, sizeof nq, cudaMemcpyDeviceToHost) != cudaSuccess) return FKK_ERR_CUDA;
    if (!b->params.pec) nq = 0;
    if (count != (size_t)nq) return FKK_ERR_INVALID_ARG;
    std::vector<int64_t> tmp(nq > 0 ? nq : 1);
    if (nq && cudaMemcpy(tmp.data(), b->q, nq * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return FKK_ERR_CUDA;
    for (int i = 0; i < nq; ++i) dst[i] = (double)tmp[i];
    return FKK_OK;
  }
  if (count != want) return FKK_ERR_INVALID_ARG;
  return cudaMemcpy(dst, src, want * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess ? FKK_OK : FKK_ERR_CUDA;
}

fkk_status fkk_gram(fkk_ctx* ctx, const float* i_cars, int64_t n, int32_t m, int64_t ld, const float* i_ref,
                    float floor_, const double* f, double* g_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!i_cars || !i_ref || !g_out || n < 1 || m < 1 || m > 2048 || ld < m || !(floor_ > 0.f))
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_gram: bad arguments");
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  DtLayout D;
  FKK_TRY(launch_transform(ctx, i_cars, n, m, ld, i_ref, floor_, D, st));
  return launch_gram(ctx, D, f, g_out, st);
}

fkk_status fkk_eig_topk(fkk_ctx* ctx, const double* g, int32_t m, int32_t k, double* lam, double* v,
                        void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!g || !lam || !v || m < 2 || m > 2048 || k < 1 || k > 80 || k > m)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_eig_topk: bad arguments");
  FKK_TRY(bind(ctx));
  return launch_eig_topk(ctx, g, m, k, lam, v, as_stream(stream));
}

fkk_status fkk_project(fkk_ctx* ctx, const float* i_cars, int64_t n, int32_t m, int64_t ld, const float* i_ref,
                       float floor_, const double* f, const double* w, int32_t k, float* p_out, int64_t* qmax,
                       int64_t* qmin, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!i_cars || !i_ref || !w || !p_out || n < 1 || m < 1 || m > 2048 || ld < m || k < 1 || k > 80 ||
      !(floor_ > 0.f) || ((qmax == nullptr) != (qmin == nullptr)))
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_project: bad arguments");
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  DtLayout D;
  FKK_TRY(launch_transform(ctx, i_cars, n, m, ld, i_ref, floor_, D, st));
  return launch_project(ctx, D, w, f, k, p_out, qmax, qmin, st);
}

fkk_status fkk_basis_math(fkk_ctx* ctx, int32_t m, int32_t k, const double* v, const double* f,
                          const double* x_rows, int32_t nq, const fkk_fit_params* params, double* c_amp,
                          double* c_ph, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!params || !v || !c_amp || !c_ph || m < 8 || m > 2048) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_basis_math: bad arguments");
  fkk_fit_params p = *params;
  p.k = k;
  if (k < 1) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_basis_math: k must be >= 1");
  FKK_TRY(check_params(ctx, p, m, k));
  if (p.pec && (!x_rows || nq < 1 || nq > 2 * k)) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_basis_math: bad x_rows / nq");
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  fkk_status s;
  int* nq_dev = (int*)workspace(ctx, "fit_nq", 64, &s);
  if (!nq_dev) return s;
  FKK_CUDA(ctx, cudaMemcpyAsync(nq_dev, &nq, sizeof(int), cudaMemcpyHostToDevice, st));
  FKK_CUDA(ctx, cudaStreamSynchronize(st));
  const int L = p.pad_len ? p.pad_len : next_pow2(2 * (int64_t)m);
  BasisOut bo{c_amp, c_ph, nullptr, nullptr, nullptr, nullptr, nullptr};
  return launch_basis_math(ctx, basis_params(p, m, L), v, f, x_rows, p.pec ? nq : 1, bo, st);
}

fkk_status fkk_reconstruct(fkk_ctx* ctx, const float* p, int64_t n, int32_t k, int32_t m, const double* c_amp,
                           const double* c_ph, float* im, float* re, int64_t ld_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!p || !c_amp || !c_ph || !im || n < 0 || k < 1 || k > 80 || m < 1 || ld_out < m)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct: bad arguments");
  if (n == 0) return FKK_OK;
  FKK_TRY(bind(ctx));
  return launch_reconstruct(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, as_stream(stream));
}

}  // extern "C"
