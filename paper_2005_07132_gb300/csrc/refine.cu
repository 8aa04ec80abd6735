// Refinement of the kept basis V_k (M x k) of the eigensolve of
// G = A^T A (Sec. 2.2 needs V and S of the SVD of A), in fp64: each step is
// one subspace iteration and a Rayleigh-Ritz projection,
//   Z = G V            (= A^T (A V), with the Gram matrix already formed)
//   Q = orth(Z)        (Cholesky QR: Z^T Z = R^T R, Q = Z R^-1)
//   H = Q^T (G Q)      (k x k)
//   H = U diag(mu) U^T (the double-word eigensolver on the k x k matrix)
//   V = Q U, lambda = mu, largest-magnitude component of each column positive.
// Exact eigenvectors come back unchanged up to rounding; an approximate basis
// gains about the eigenvalue gap ratio lambda_{k+1} / lambda_k per step.
#include "common.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr int kT = 32;  // output tile (rows of G x columns of V) and K chunk

// out (m x k, row-major) = G (m x m, row-major) V (m x k, row-major), fp64;
// a 256-thread block computes a 32 x 32 tile, 4 outputs per thread.
__global__ void __launch_bounds__(256) gv_kernel(const double* __restrict__ g, const double* __restrict__ v, int m,
                                                 int k, double* __restrict__ out) {
  __shared__ double gs[kT][kT + 1];
  __shared__ double vs[kT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7: rows ty, ty + 8, ty + 16, ty + 24
  const int i0 = blockIdx.x * kT, c0 = blockIdx.y * kT;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j0 = 0; j0 < m; j0 += kT) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int li = ty + 8 * r;
      const int i = i0 + li, j = j0 + tx;
      gs[li][tx] = (i < m && j < m) ? g[(size_t)i * m + j] : 0.0;
      const int jj = j0 + li, c = c0 + tx;
      vs[li][tx] = (jj < m && c < k) ? v[(size_t)jj * k + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < kT; ++q) {
      const double vq = vs[q][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(gs[ty + 8 * r][q], vq, acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 8 * r, c = c0 + tx;
    if (i < m && c < k) out[(size_t)i * k + c] = acc[r];
  }
}

// h (k x k) = Q^T X for Q, X m x k row-major: one block per entry.
__global__ void __launch_bounds__(128) atb_kernel(const double* __restrict__ q, const double* __restrict__ x, int m,
                                                  int k, double* __restrict__ h) {
  const int a = blockIdx.x, b = blockIdx.y;
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) acc = fma(q[(size_t)i * k + a], x[(size_t)i * k + b], acc);
  acc = warp_sum(acc);
  __shared__ double red[4];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) h[a * k + b] = (red[0] + red[1]) + (red[2] + red[3]);
}

// h <- (h + h^T) / 2 (the Rayleigh quotient is symmetric; rounding is not)
__global__ void symmetrize_kernel(double* __restrict__ h, int k) {
  const int a = blockIdx.x, b = threadIdx.x;
  if (b >= k || b <= a) return;
  const double s = 0.5 * (h[a * k + b] + h[b * k + a]);
  h[a * k + b] = s;
  h[b * k + a] = s;
}

// v (m x k) = Q (m x k) U (k x k), all row-major
__global__ void qu_kernel(const double* __restrict__ q, const double* __restrict__ u, int m, int k,
                          double* __restrict__ v) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * k) return;
  const int i = (int)(t / k), c = (int)(t % k);
  double acc = 0.0;
  for (int a = 0; a < k; ++a) acc = fma(q[(size_t)i * k + a], u[(size_t)a * k + c], acc);
  v[t] = acc;
}

// k = 1: the 1 x 1 Rayleigh quotient is its own eigenvalue, U = 1
__global__ void one_by_one_kernel(const double* __restrict__ h, double* __restrict__ mu, double* __restrict__ u) {
  mu[0] = h[0];
  u[0] = 1.0;
}

fkk_status gv(fkk_ctx* ctx, const double* g, const double* v, int m, int k, double* out, cudaStream_t st) {
  FKK_COUNT_LAUNCH();
  gv_kernel<<<dim3((m + kT - 1) / kT, (k + kT - 1) / kT), 256, 0, st>>>(g, v, m, k, out);
  return cuda_check(ctx, cudaGetLastError(), "refine: G V");
}

}  // namespace

fkk_status launch_refine(fkk_ctx* ctx, const double* g, int m, int k, const double* v_in, int steps, double* lam,
                         double* v_out, cudaStream_t st) {
  if (steps < 1) return FKK_OK;
  if (k < 1 || k > m || k > 80) return fail(ctx, FKK_ERR_INVALID_ARG, "refine: k = %d", k);
  fkk_status s;
  const size_t mk = (size_t)m * k * sizeof(double), kk = (size_t)k * k * sizeof(double);
  double* z = (double*)workspace(ctx, "ref_z", mk, &s);
  if (!z) return s;
  double* q = (double*)workspace(ctx, "ref_q", mk, &s);
  if (!q) return s;
  double* h = (double*)workspace(ctx, "ref_h", kk, &s);
  if (!h) return s;
  double* u = (double*)workspace(ctx, "ref_u", kk, &s);
  if (!u) return s;
  double* w = (double*)workspace(ctx, "ref_w", 2 * kk, &s);
  if (!w) return s;
  const double* cur = v_in;
  for (int step = 0; step < steps; ++step) {
    FKK_TRY(gv(ctx, g, cur, m, k, z, st));                          // Z = G V
    FKK_TRY(launch_ztz(ctx, z, m, k, w, st));                       // Z^T Z
    FKK_TRY(launch_chol_inv(ctx, w, k, w + (size_t)k * k, st, 1e-20, true));
    FKK_TRY(launch_apply_rinv(ctx, z, m, k, w + (size_t)k * k, q, st));  // Q = Z R^-1
    FKK_TRY(gv(ctx, g, q, m, k, z, st));                            // G Q
    FKK_COUNT_LAUNCH();
    atb_kernel<<<dim3(k, k), 128, 0, st>>>(q, z, m, k, h);          // H = Q^T G Q
    FKK_COUNT_LAUNCH();
    symmetrize_kernel<<<k, ((k + 31) / 32) * 32, 0, st>>>(h, k);
    FKK_CUDA(ctx, cudaGetLastError());
    if (k == 1) {
      FKK_COUNT_LAUNCH();
      one_by_one_kernel<<<1, 1, 0, st>>>(h, lam, u);
      FKK_CUDA(ctx, cudaGetLastError());
    } else {
      FKK_TRY(launch_eig_topk(ctx, h, k, k, lam, u, st));             // H = U diag(mu) U^T
    }
    FKK_COUNT_LAUNCH();
    qu_kernel<<<(unsigned)(((int64_t)m * k + 255) / 256), 256, 0, st>>>(q, u, m, k, v_out);  // V = Q U
    FKK_CUDA(ctx, cudaGetLastError());
    cur = v_out;
  }
  return launch_sign_fix(ctx, v_out, m, k, st);
}

}  // namespace fkk

using namespace fkk;

extern "C" fkk_status fkk_refine_basis(fkk_ctx* ctx, const double* g, int32_t m, int32_t k, const double* v,
                                       int32_t steps, double* lam_out, double* v_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!g || !v || !lam_out || !v_out || m < 2 || m > 2048 || k < 1 || k > 80 || k > m || steps < 1 || steps > 4)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_refine_basis: bad arguments");
  FKK_TRY(bind(ctx));
  return launch_refine(ctx, g, m, k, v, steps, lam_out, v_out, as_stream(stream));
}
