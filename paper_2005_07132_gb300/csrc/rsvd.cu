// Randomised SVD of the transformed cube (Sec. 5 proposes a randomised SVD
// for fast retraining; Halko, Martinsson & Tropp 2011, randomised subspace
// iteration):
//   Omega (m x l): Philox4x64-10 Gaussians, l = k + oversample
//   Y = A Omega;  repeat power_iters times: Q = orth(Y), Z = orth(A^T Q),
//   Y = A Z;  Q = orth(Y);  B^T = A^T Q (m x l)
//   B B^T = U diag(s^2) U^T (l x l),  V = B^T U diag(1/s)
// A never exists: A X is the tensor-core projection of the transformed cube
// (its shift c folded in), A^T Q the Gram kernel with Q^T as its second
// operand.  orth() of the tall N x l matrices is Cholesky QR twice, with fp32
// products summed in fp64 per block and over blocks in a fixed order; the
// small m x l ones use the eigensolver's fp64 Cholesky QR.
#include <algorithm>

#include "common.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr uint64_t kPhM0 = 0xD2E7470EE14C6C93ull, kPhM1 = 0xCA5A826395121157ull;  // multipliers
constexpr uint64_t kPhW0 = 0x9E3779B97F4A7C15ull, kPhW1 = 0xBB67AE8584CAA73Bull;  // key increments

// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11) on counter c, key (k0, k1).
__device__ __forceinline__ void philox4x64_10(uint64_t (&c)[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(kPhM0, c[0]), lo0 = kPhM0 * c[0];
    const uint64_t hi1 = __umul64hi(kPhM1, c[2]), lo1 = kPhM1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += kPhW0;
    k1 += kPhW1;
  }
}

// out[e], e < count: counter (e / 2, 0, 0, 0), key (seed, 0); words 0 and 1
// give u = ((w >> 11) + 1/2) 2^-53; Box-Muller: sqrt(-2 ln u1) cos(2 pi u2)
// for even e, sin for odd e.
__global__ void philox_normal_kernel(int64_t count, uint64_t seed, double* __restrict__ out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * b >= count) return;
  uint64_t c[4] = {(uint64_t)b, 0, 0, 0};
  philox4x64_10(c, seed, 0);
  const double u1 = ((double)(c[0] >> 11) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)(c[1] >> 11) + 0.5) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  out[2 * b] = r * cs;
  if (2 * b + 1 < count) out[2 * b + 1] = r * sn;
}

constexpr int kMaxL = 80;
constexpr int kTallThreads = 256;  // a 16 x 16 grid of T x T output tiles
constexpr int kTallRows = 32;      // rows per shared-memory tile
constexpr int kTallFlush = 4;      // tiles summed in fp32 before each fp64 add

// Block b: partial[b][p * lp + q] = sum over its rows of x[r][p] x[r][q]
// (lp = 16 T >= l, the full square).  Each thread owns a T x T tile of
// (p, q); products in fp32 over kTallFlush tiles of 32 rows, then fp64.
template <int T>
__global__ void __launch_bounds__(kTallThreads) gram_tall_kernel(const float* __restrict__ x, int64_t n, int l,
                                                                 int64_t rows_per_block,
                                                                 double* __restrict__ partial) {
  constexpr int lp = 16 * T;
  constexpr int ls = lp + 4;  // row stride: 16-byte aligned, rows offset by 4 banks
  __shared__ __align__(16) float tile[kTallRows][ls];
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  float a32[T][T];
  double acc[T][T];
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) {
      a32[a][b] = 0.f;
      acc[a][b] = 0.0;
    }
  int ntile = 0;
  for (int64_t base = r0; base < r1; base += kTallRows) {
    __syncthreads();
    for (int e = threadIdx.x; e < kTallRows * lp; e += kTallThreads) {
      const int rr = e / lp, cc = e - rr * lp;
      const int64_t r = base + rr;
      tile[rr][cc] = (r < r1 && cc < l) ? x[r * l + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kTallRows; ++rr) {
      float xp[T], xq[T];
      if constexpr (T == 4) {
        const float4 u = *reinterpret_cast<const float4*>(&tile[rr][ty * 4]);
        const float4 v = *reinterpret_cast<const float4*>(&tile[rr][tx * 4]);
        xp[0] = u.x; xp[1] = u.y; xp[2] = u.z; xp[3] = u.w;
        xq[0] = v.x; xq[1] = v.y; xq[2] = v.z; xq[3] = v.w;
      } else {
#pragma unroll
        for (int a = 0; a < T; ++a) {
          xp[a] = tile[rr][ty * T + a];
          xq[a] = tile[rr][tx * T + a];
        }
      }
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) a32[a][b] = fmaf(xp[a], xq[b], a32[a][b]);
    }
    if (++ntile == kTallFlush) {
      ntile = 0;
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) {
          acc[a][b] += a32[a][b];
          a32[a][b] = 0.f;
        }
    }
  }
  double* out = partial + (int64_t)blockIdx.x * lp * lp;
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b)
      out[(ty * T + a) * lp + tx * T + b] = acc[a][b] + a32[a][b];
}

// g (l x l) = sum of the partials (lp x lp each) in block order: a block per
// entry, a fixed-order tree over the partials.
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nblocks, int l, int lp,
                                   double* __restrict__ g) {
  __shared__ double red[32];
  const int e = blockIdx.x, p = e / l, q = e - p * l;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)b * lp * lp + p * lp + q];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g[e] = t;
  }
}

// Rows r0 = 64 b .. r0 + 63: q = x R^-1 (R^-1 upper triangular, used in
// fp32) as a small GEMM, each thread a 4 x 4 tile of (row, column) (a 16 x 16
// thread grid over 64 rows x 64 columns; l <= 64 here, wider sketches run
// the columns in two passes).  Writes q (row-major, if q_out), and / or Q^T in
// bf16 hi / lo at [c][np] (zero for rows >= n) with per-block column sums.
constexpr int kApRows = 64;
constexpr int kApCols = 64;  // columns per pass
__global__ void __launch_bounds__(256) apply_rinv_tall_kernel(const float* __restrict__ x, int64_t n, int l,
                                                              const double* __restrict__ rinv,
                                                              float* __restrict__ q_out,
                                                              __nv_bfloat16* __restrict__ qt_hi,
                                                              __nv_bfloat16* __restrict__ qt_lo, int64_t np,
                                                              double* __restrict__ colsum_part) {
  extern __shared__ __align__(16) float ap_sm[];
  constexpr int xs_ld = kMaxL + 4, rs_ld = kApCols + 4, qs_ld = kApRows + 1;
  float* xs = ap_sm;                      // [kApRows][xs_ld]: x, transposed access by column p
  float* rs = xs + kApRows * xs_ld;       // [kMaxL][rs_ld]: R^-1 rows p, this pass's columns
  float* qs = rs + kMaxL * rs_ld;         // [kMaxL][qs_ld]: q^T
  const int64_t r0 = (int64_t)blockIdx.x * kApRows;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int e = threadIdx.x; e < kApRows * l; e += blockDim.x) {
    const int rr = e / l, cc = e - rr * l;
    const int64_t r = r0 + rr;
    xs[rr * xs_ld + cc] = r < n ? x[r * l + cc] : 0.f;
  }
  for (int c0 = 0; c0 < l; c0 += kApCols) {
    __syncthreads();
    for (int e = threadIdx.x; e < l * kApCols; e += blockDim.x) {
      const int p = e / kApCols, c = c0 + (e - p * kApCols);
      rs[p * rs_ld + (c - c0)] = (c < l && p <= c) ? (float)rinv[p * l + c] : 0.f;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int p = 0; p < l; ++p) {
      float xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = xs[(ty * 4 + a) * xs_ld + p];
      const float4 rv = *reinterpret_cast<const float4*>(&rs[p * rs_ld + tx * 4]);
      const float rr4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xv[a], rr4[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int rr = ty * 4 + a;
      const int64_t r = r0 + rr;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + tx * 4 + b;
        if (c < l) {
          const float v = r < n ? acc[a][b] : 0.f;
          if (q_out && r < n) q_out[r * l + c] = v;
          qs[c * qs_ld + rr] = v;
        }
      }
    }
  }
  __syncthreads();
  if (qt_hi) {
    for (int e = threadIdx.x; e < l * (kApRows / 2); e += blockDim.x) {
      const int cc = e / (kApRows / 2), pr = e - cc * (kApRows / 2);
      __nv_bfloat16 ah, al, bh, bl;
      split_bf16(qs[cc * qs_ld + 2 * pr], ah, al);
      split_bf16(qs[cc * qs_ld + 2 * pr + 1], bh, bl);
      const int64_t off = (int64_t)cc * np + r0 + 2 * pr;
      *reinterpret_cast<__nv_bfloat162*>(qt_hi + off) = __halves2bfloat162(ah, bh);
      *reinterpret_cast<__nv_bfloat162*>(qt_lo + off) = __halves2bfloat162(al, bl);
    }
  }
  if (colsum_part)
    for (int cc = threadIdx.x; cc < l; cc += blockDim.x) {
      double sum = 0.0;
      for (int rr = 0; rr < kApRows; ++rr) sum += qs[cc * qs_ld + rr];
      colsum_part[(int64_t)blockIdx.x * l + cc] = sum;
    }
}

constexpr size_t kApSmem =
    sizeof(float) * ((size_t)kApRows * (kMaxL + 4) + (size_t)kMaxL * (kApCols + 4) + (size_t)kMaxL * (kApRows + 1));

// out[c] = sum of the per-block column sums: a block per column, a
// fixed-order tree.
__global__ void colsum_reduce_kernel(const double* __restrict__ part, int nblocks, int l, double* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(int64_t)b * l + c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[c] = t;
  }
}

// V[j, i] = sum_p Z[j, p] U[p, i] / sqrt(lam[i]) (Z = B^T, m x l; U l x k).
__global__ void bu_kernel(const double* __restrict__ z, int m, int l, const double* __restrict__ u,
                          const double* __restrict__ lam, int k, double* __restrict__ v) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * k) return;
  const int j = (int)(t / k), i = (int)(t - (int64_t)j * k);
  double s = 0.0;
  for (int p = 0; p < l; ++p) s = fma(z[(int64_t)j * l + p], u[(int64_t)p * k + i], s);
  const double sv = sqrt(fmax(lam[i], 0.0));
  v[t] = sv > 0.0 ? s / sv : 0.0;
}

}  // namespace

fkk_status launch_rsvd(fkk_ctx* ctx, const DtLayout& L, const double* f, int k, int oversample, int power_iters,
                       uint64_t seed, double* lam, double* v, cudaStream_t st) {
  const int m = L.m;
  const int64_t n = L.n, np = L.np;
  const int l = std::min(k + oversample, m);
  if (k < 1 || l < k || l > kMaxL || power_iters < 0)
    return fail(ctx, FKK_ERR_INVALID_ARG, "randomised SVD: k = %d, l = %d (at most %d)", k, l, kMaxL);
  const int tn = l <= 64 ? 64 : 128;
  const int tt = l <= 64 ? 4 : 5, lp = 16 * tt;
  int gblocks = (int)std::min<int64_t>((int64_t)ctx->sm_count * 8, (n + kTallRows - 1) / kTallRows);
  if (gblocks < 1) gblocks = 1;
  const int64_t rows_per_block = (n + gblocks - 1) / gblocks;
  const int ablocks = (int)(np / kApRows);
  fkk_status s;
  auto ws = [&](const char* name, size_t bytes) { return workspace(ctx, name, bytes, &s); };
  double* om = (double*)ws("rsvd_omega", (size_t)m * l * 8);
  float* y = om ? (float*)ws("rsvd_y", (size_t)n * l * 4) : nullptr;
  float* q1 = y ? (float*)ws("rsvd_q1", (size_t)n * l * 4) : nullptr;
  __nv_bfloat16* qt = q1 ? (__nv_bfloat16*)ws("rsvd_qt", (size_t)2 * tn * np * 2) : nullptr;
  double* small = qt ? (double*)ws("rsvd_small", (size_t)(4 * m * l + 4 * l * l + l * k + 2 * l) * 8) : nullptr;
  double* gpart = small ? (double*)ws("rsvd_gpart", (size_t)gblocks * lp * lp * 8) : nullptr;
  double* cpart = gpart ? (double*)ws("rsvd_cpart", (size_t)ablocks * l * 8) : nullptr;
  if (!cpart) return s;
  __nv_bfloat16* qt_hi = qt;
  __nv_bfloat16* qt_lo = qt + (size_t)tn * np;
  double* z = small;                 // m x l: A^T Q
  double* zo = z + (size_t)m * l;    // m x l: orth(A^T Q)
  double* zt = zo + (size_t)m * l;   // m x l: scratch for the second QR pass
  double* g = zt + (size_t)m * l;    // l x l
  double* rinv = g + (size_t)l * l;  // l x l
  double* c = rinv + (size_t)l * l;  // l x l: B B^T
  double* u = c + (size_t)l * l;     // l x k
  double* colsum = u + (size_t)l * k;
  FKK_CUDA(ctx, cudaMemsetAsync(qt, 0, (size_t)2 * tn * np * 2, st));
  FKK_CUDA(ctx, cudaFuncSetAttribute(apply_rinv_tall_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApSmem));

  // Q^T hi / lo and its column sums from the tall Y by Cholesky QR: one pass
  // while the power iterations only need the span, two for the final Q
  auto orth_tall = [&](int passes) -> fkk_status {
    for (int pass = 0; pass < passes; ++pass) {
      const float* src = pass == 0 ? y : q1;
      FKK_COUNT_LAUNCH();
      if (tt == 4)
        gram_tall_kernel<4><<<gblocks, kTallThreads, 0, st>>>(src, n, l, rows_per_block, gpart);
      else
        gram_tall_kernel<5><<<gblocks, kTallThreads, 0, st>>>(src, n, l, rows_per_block, gpart);
      FKK_COUNT_LAUNCH();
      gram_reduce_kernel<<<l * l, 128, 0, st>>>(gpart, gblocks, l, lp, g);
      FKK_CUDA(ctx, cudaGetLastError());
      // the Gram's fp32 products resolve about 1e-7 of the largest column's
      // squared norm: a column below 1e-6 of its own is taken as dependent
      FKK_TRY(launch_chol_inv(ctx, g, l, rinv, st, 1e-6, false));
      const bool last = pass == passes - 1;
      FKK_COUNT_LAUNCH();
      apply_rinv_tall_kernel<<<ablocks, 256, kApSmem, st>>>(src, n, l, rinv, last ? nullptr : q1,
                                                            last ? qt_hi : nullptr, qt_lo, np,
                                                            last ? cpart : nullptr);
      FKK_CUDA(ctx, cudaGetLastError());
    }
    FKK_COUNT_LAUNCH();
    colsum_reduce_kernel<<<l, 256, 0, st>>>(cpart, ablocks, l, colsum);
    return cuda_check(ctx, cudaGetLastError(), "randomised SVD: orth");
  };

  FKK_COUNT_LAUNCH();
  philox_normal_kernel<<<(unsigned)(((int64_t)m * l / 2 + 1 + 255) / 256), 256, 0, st>>>((int64_t)m * l, seed, om);
  FKK_CUDA(ctx, cudaGetLastError());
  FKK_TRY(launch_project_tc(ctx, L, om, f, l, y, nullptr, st));  // Y = A Omega
  for (int it = 0;; ++it) {
    FKK_TRY(orth_tall(it == power_iters ? 2 : 1));
    FKK_TRY(launch_atq(ctx, L, qt_hi, qt_lo, tn, l, colsum, f, z, st));  // A^T Q
    if (it == power_iters) break;
    // Z = orth(A^T Q) in fp64 (its span is what the next step needs), Y = A Z
    FKK_TRY(launch_ztz(ctx, z, m, l, g, st));
    FKK_TRY(launch_chol_inv(ctx, g, l, rinv, st, 1e-20, false));
    FKK_TRY(launch_apply_rinv(ctx, z, m, l, rinv, zo, st));
    FKK_TRY(launch_project_tc(ctx, L, zo, f, l, y, nullptr, st));
  }
  // B^T = A^T Q; B B^T = Z^T Z; its k leading eigenpairs give s^2 and U
  FKK_TRY(launch_ztz(ctx, z, m, l, c, st));
  FKK_TRY(launch_eig_topk(ctx, c, l, k, lam, u, st));
  FKK_COUNT_LAUNCH();
  bu_kernel<<<(unsigned)(((int64_t)m * k + 255) / 256), 256, 0, st>>>(z, m, l, u, lam, k, v);
  FKK_CUDA(ctx, cudaGetLastError());
  return launch_sign_fix(ctx, v, m, k, st);
}

}  // namespace fkk

using namespace fkk;

extern "C" fkk_status fkk_philox_normals(fkk_ctx* ctx, int64_t count, uint64_t seed, double* out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (count < 0 || (count > 0 && !out)) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_philox_normals: bad arguments");
  if (count == 0) return FKK_OK;
  FKK_TRY(bind(ctx));
  FKK_COUNT_LAUNCH();
  philox_normal_kernel<<<(unsigned)((count / 2 + 1 + 255) / 256), 256, 0, as_stream(stream)>>>(count, seed, out);
  return cuda_check(ctx, cudaGetLastError(), "fkk_philox_normals");
}
