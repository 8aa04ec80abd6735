// Projection of the spectra on the basis: P = A W = U S (W = V for the fit,
// W = V diag(s^2/(s^2+lambda)) for new data, Eq. ML_Unew), with the per-
// column argmax / argmin rows that form the fPEC sub-sample q (Eqs. q_max,
// q_min).  One thread owns one spectrum and all k outputs; the basis is
// staged through shared memory in 128-channel chunks.
#include "common.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr int kRows = 128;   // spectra per block (one per thread)
constexpr int kChunk = 128;  // channels per shared-memory chunk

struct ProjArgs {
  const __nv_bfloat16* dt_hi;
  const __nv_bfloat16* dt_lo;
  int64_t np;
  const float* i_cars;  // raw path
  int64_t ld;
  const float* i_ref;
  float floor_;
  int64_t n;
  int m;
  int k;
  const float* wf;   // m x k fp32: f * W
  const float* off;  // k: c^T (f W) (transformed path only)
  float* p;          // n x k
  float4* cand;      // per block, per column: (max, argmax, min, argmin)
  long long* status;
};

// KC: k rounded up to a multiple of 8 (compile-time accumulator count)
template <int KC, bool RAW>
__global__ void __launch_bounds__(kRows) project_kernel(ProjArgs a) {
  __shared__ float wsm[kChunk][KC];
  __shared__ float redv[4][KC][2];
  __shared__ int redi[4][KC][2];
  const int tid = threadIdx.x;
  const int64_t n = (int64_t)blockIdx.x * kRows + tid;
  const bool valid = n < a.n;
  float acc[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) acc[i] = 0.f;
  int clamped = 0;
  for (int j0 = 0; j0 < a.m; j0 += kChunk) {
    const int cw = min(kChunk, a.m - j0);
    __syncthreads();
    for (int t = tid; t < kChunk * KC; t += kRows) {
      int jj = t / KC, i = t % KC;
      wsm[jj][i] = (jj < cw && i < a.k) ? a.wf[(int64_t)(j0 + jj) * a.k + i] : 0.f;
    }
    __syncthreads();
    if (valid) {
      for (int jj = 0; jj < cw; ++jj) {
        const int j = j0 + jj;
        float d;
        if (RAW) {
          float x = a.i_cars[n * a.ld + j] / a.i_ref[j];
          if (!(x >= a.floor_)) { x = a.floor_; ++clamped; }
          d = 0.5f * logf(x);
        } else {
          const int64_t o = (int64_t)j * a.np + n;
          d = __bfloat162float(a.dt_hi[o]) + __bfloat162float(a.dt_lo[o]);
        }
#pragma unroll
        for (int i = 0; i < KC; ++i) acc[i] = fmaf(d, wsm[jj][i], acc[i]);
      }
    }
  }
  if (!RAW) {
#pragma unroll
    for (int i = 0; i < KC; ++i) acc[i] += (i < a.k) ? a.off[i] : 0.f;
  }
  if (valid) {
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < a.k) a.p[n * a.k + i] = acc[i];
  }
  if (RAW) {
    for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
    if ((tid & 31) == 0 && clamped)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.status + 1), (unsigned long long)clamped);
    return;
  }
  if (!a.cand) return;
  // per-column (max, argmax, min, argmin) over the block, ties to the lowest row
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int i = 0; i < KC; ++i) {
    float mx = valid ? acc[i] : -INFINITY, mn = valid ? acc[i] : INFINITY;
    int imx = valid ? (int)n : 0x7fffffff, imn = imx;
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, mx, o);
      int oi = __shfl_xor_sync(0xffffffffu, imx, o);
      if (ov > mx || (ov == mx && oi < imx)) { mx = ov; imx = oi; }
      ov = __shfl_xor_sync(0xffffffffu, mn, o);
      oi = __shfl_xor_sync(0xffffffffu, imn, o);
      if (ov < mn || (ov == mn && oi < imn)) { mn = ov; imn = oi; }
    }
    if (lane == 0) {
      redv[warp][i][0] = mx; redi[warp][i][0] = imx;
      redv[warp][i][1] = mn; redi[warp][i][1] = imn;
    }
  }
  __syncthreads();
  if (tid < a.k) {
    const int i = tid;
    float mx = redv[0][i][0], mn = redv[0][i][1];
    int imx = redi[0][i][0], imn = redi[0][i][1];
    for (int w = 1; w < 4; ++w) {
      float v = redv[w][i][0]; int q = redi[w][i][0];
      if (v > mx || (v == mx && q < imx)) { mx = v; imx = q; }
      v = redv[w][i][1]; q = redi[w][i][1];
      if (v < mn || (v == mn && q < imn)) { mn = v; imn = q; }
    }
    a.cand[(int64_t)blockIdx.x * a.k + i] = make_float4(mx, __int_as_float(imx), mn, __int_as_float(imn));
  }
}

// Reduce block candidates in block order: qmax[i], qmin[i].
__global__ void argext_reduce_kernel(const float4* __restrict__ cand, int nblocks, int k, int64_t* qmax,
                                     int64_t* qmin) {
  const int i = blockIdx.x;
  float mx = -INFINITY, mn = INFINITY;
  int imx = 0x7fffffff, imn = 0x7fffffff;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    float4 c = cand[(int64_t)b * k + i];
    int q0 = __float_as_int(c.y), q1 = __float_as_int(c.w);
    if (c.x > mx || (c.x == mx && q0 < imx)) { mx = c.x; imx = q0; }
    if (c.z < mn || (c.z == mn && q1 < imn)) { mn = c.z; imn = q1; }
  }
  __shared__ float sv[2][32];
  __shared__ int si[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, mx, o);
    int oi = __shfl_xor_sync(0xffffffffu, imx, o);
    if (ov > mx || (ov == mx && oi < imx)) { mx = ov; imx = oi; }
    ov = __shfl_xor_sync(0xffffffffu, mn, o);
    oi = __shfl_xor_sync(0xffffffffu, imn, o);
    if (ov < mn || (ov == mn && oi < imn)) { mn = ov; imn = oi; }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sv[0][w] = mx; si[0][w] = imx; sv[1][w] = mn; si[1][w] = imn; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      if (sv[0][q] > mx || (sv[0][q] == mx && si[0][q] < imx)) { mx = sv[0][q]; imx = si[0][q]; }
      if (sv[1][q] < mn || (sv[1][q] == mn && si[1][q] < imn)) { mn = sv[1][q]; imn = si[1][q]; }
    }
    // also the values gathered by thread 0 itself were included above via the shuffle
    qmax[i] = imx;
    qmin[i] = imn;
  }
}

// wf[j, i] = f_j W[j, i] (fp32) and off[i] = sum_j c_j wf[j, i] (c may be null)
__global__ void prep_w_kernel(const double* __restrict__ w, const double* __restrict__ f, const float* __restrict__ c,
                              int m, int k, float* __restrict__ wf, float* __restrict__ off) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double v = w[(int64_t)j * k + i] * (f ? f[j] : 1.0);
    wf[(int64_t)j * k + i] = (float)v;
    if (c) acc += (double)c[j] * v;
  }
  if (!off) return;
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    off[i] = (float)s;
  }
}

template <bool RAW>
fkk_status dispatch_project(fkk_ctx* ctx, ProjArgs& a, unsigned grid, cudaStream_t st) {
  switch ((a.k + 7) / 8) {
#define FKK_PROJ_CASE(KB) \
  case KB: FKK_COUNT_LAUNCH(); project_kernel<KB * 8, RAW><<<grid, kRows, 0, st>>>(a); break;
    FKK_PROJ_CASE(1)
    FKK_PROJ_CASE(2)
    FKK_PROJ_CASE(3)
    FKK_PROJ_CASE(4)
    FKK_PROJ_CASE(5)
    FKK_PROJ_CASE(6)
    FKK_PROJ_CASE(7)
    FKK_PROJ_CASE(8)
    FKK_PROJ_CASE(9)
    FKK_PROJ_CASE(10)
#undef FKK_PROJ_CASE
    default:
      return fail(ctx, FKK_ERR_INVALID_ARG, "k=%d outside 1..80", a.k);
  }
  return cuda_check(ctx, cudaGetLastError(), "project_kernel launch");
}

}  // namespace

fkk_status launch_project(fkk_ctx* ctx, const DtLayout& L, const double* w, const double* f, int k, float* p,
                          int64_t* qmax, int64_t* qmin, cudaStream_t st) {
  fkk_status s;
  const unsigned grid = (unsigned)((L.n + kRows - 1) / kRows);  // 128-row tiles
  float4* cand = nullptr;
  if (qmax) {
    cand = (float4*)workspace(ctx, "proj_cand", (size_t)grid * k * sizeof(float4), &s);
    if (!cand) return s;
  }
  FKK_TRY(launch_project_tc(ctx, L, w, f, k, p, cand, st));
  if (qmax) {
    FKK_COUNT_LAUNCH(); argext_reduce_kernel<<<k, 256, 0, st>>>(cand, (int)grid, k, qmax, qmin);
    FKK_CUDA(ctx, cudaGetLastError());
  }
  return FKK_OK;
}

fkk_status launch_project_raw(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                              const float* i_ref, float floor_, const double* w, const double* f, int k,
                              float* p, cudaStream_t st) {
  fkk_status s;
  float* wf = (float*)workspace(ctx, "projraw_wf", (size_t)m * k * 4, &s);
  if (!wf) return s;
  FKK_COUNT_LAUNCH(); prep_w_kernel<<<k, 256, 0, st>>>(w, f, nullptr, m, k, wf, nullptr);
  const unsigned grid = (unsigned)((n + kRows - 1) / kRows);
  ProjArgs a{nullptr, nullptr, 0, i_cars, ld, i_ref, floor_, n, m, k, wf, nullptr, p, nullptr, ctx->d_status};
  return dispatch_project<true>(ctx, a, grid, st);
}

}  // namespace fkk
