// Transform pass of the fit: d = 1/2 ln(max(I/I_ref, floor)) - c (or, in
// raw mode for the conventional workflow's SVD denoising, d = I - c), stored
// channel-major as two bf16 terms (D^T_hi, D^T_lo), plus per-channel sums of
// d and of I.  c is a per-channel shift (the mean log ratio of the first
// rows); it leaves A^T A unchanged in exact arithmetic,
//   sum_n a a^T = sum_n d d^T + s c^T + c s^T + N c c^T,  s = sum_n d,
// while shrinking the magnitudes the tensor-core Gram accumulates.
#include "common.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr int kShiftRows = 256;

__global__ void shift_kernel(const float* __restrict__ i_cars, int64_t n, int m, int64_t ld,
                             const float* __restrict__ i_ref, float floor_, float* __restrict__ c, int raw) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  int rows = (int)(n < kShiftRows ? n : kShiftRows);
  double acc = 0.0;
  if (raw) {
    for (int t = 0; t < rows; ++t) acc += i_cars[(int64_t)t * ld + j];
  } else {
    const float r = i_ref[j];
    for (int t = 0; t < rows; ++t) {
      float x = i_cars[(int64_t)t * ld + j] / r;
      x = (x >= floor_) ? x : floor_;
      acc += 0.5f * logf(x);
    }
  }
  c[j] = rows ? (float)(acc / rows) : 0.f;
}

// Block = 256 threads, tile = 64 rows x 64 channels; blockIdx.y = channel
// tile; blockIdx.x walks row tiles rt = blockIdx.x, +gridDim.x, ...
// kRaw: d = I - c (raw spectra; i_ref and the floor are not used).
template <bool kRaw>
__global__ void __launch_bounds__(256) transform_kernel(TransformArgs p) {
  __shared__ float tile[64][65];
  __shared__ double red_d[4][64];
  __shared__ double red_d2[4][64];
  __shared__ double red_i[4][64];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int j0 = blockIdx.y * 64;
  const int j = j0 + tx;
  const bool jvalid = j < p.m;
  const float rinv = (jvalid && !kRaw) ? 1.f / p.i_ref[j] : 1.f;
  const float cj = jvalid ? p.c[j] : 0.f;
  const int64_t nrt = p.np / 64;
  double sum_d = 0.0, sum_i = 0.0, sum_d2 = 0.0;
  int clamped = 0;
  for (int64_t rt = blockIdx.x; rt < nrt; rt += gridDim.x) {
    const int64_t n0 = rt * 64;
    float td = 0.f, ti = 0.f, td2 = 0.f;
    // all 16 loads of this thread in flight before any arithmetic
    float vals[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int64_t n = n0 + ty + 4 * u;
      vals[u] = (jvalid && n < p.n) ? __ldcs(p.i_cars + n * p.ld + j) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int rr = ty + 4 * u;
      const int64_t n = n0 + rr;
      float d = 0.f;
      if (jvalid && n < p.n) {
        const float v = vals[u];
        if (kRaw) {
          d = v - cj;
        } else {
          float x = v * rinv;
          if (!(x >= p.floor_)) { x = p.floor_; ++clamped; }
          d = 0.5f * logf(x) - cj;
        }
        td += d;
        td2 = fmaf(d, d, td2);
        ti += v;
      }
      tile[tx][rr] = d;
    }
    sum_d += td;
    sum_d2 += td2;
    sum_i += ti;
    __syncthreads();
    // transposed write: warp w handles channels w, w+8, ..., 32 lanes x 2 bf16
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int cc = w; cc < 64; cc += 8) {
      float a = tile[cc][2 * lane], b = tile[cc][2 * lane + 1];
      __nv_bfloat16 ah, al, bh, bl;
      split_bf16(a, ah, al);
      split_bf16(b, bh, bl);
      int64_t off = (int64_t)(j0 + cc) * p.np + n0 + 2 * lane;
      *reinterpret_cast<__nv_bfloat162*>(p.dt_hi + off) = __halves2bfloat162(ah, bh);
      *reinterpret_cast<__nv_bfloat162*>(p.dt_lo + off) = __halves2bfloat162(al, bl);
    }
    __syncthreads();
  }
  red_d[ty][tx] = sum_d;
  red_d2[ty][tx] = sum_d2;
  red_i[ty][tx] = sum_i;
  __syncthreads();
  if (ty == 0 && jvalid) {
    double sd = red_d[0][tx] + red_d[1][tx] + red_d[2][tx] + red_d[3][tx];
    double si = red_i[0][tx] + red_i[1][tx] + red_i[2][tx] + red_i[3][tx];
    p.part_d[(int64_t)blockIdx.x * p.m + j] = sd;
    p.part_d2[(int64_t)blockIdx.x * p.m + j] = red_d2[0][tx] + red_d2[1][tx] + red_d2[2][tx] + red_d2[3][tx];
    p.part_i[(int64_t)blockIdx.x * p.m + j] = si;
  }
  for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
  if ((threadIdx.x & 31) == 0 && clamped)
    atomicAdd(reinterpret_cast<unsigned long long*>(p.status + 1), (unsigned long long)clamped);
}

__global__ void colsum_reduce_kernel(const double* __restrict__ part_d, const double* __restrict__ part_i,
                                     const double* __restrict__ part_d2, int nparts, int m,
                                     double* __restrict__ sum_d, double* __restrict__ sum_i,
                                     double* __restrict__ sum_d2) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double a = 0.0, b = 0.0, c2 = 0.0;
  for (int t = 0; t < nparts; ++t) {
    a += part_d[(int64_t)t * m + j];
    b += part_i[(int64_t)t * m + j];
    c2 += part_d2[(int64_t)t * m + j];
  }
  sum_d[j] = a;
  sum_i[j] = b;
  sum_d2[j] = c2;
}

}  // namespace

fkk_status launch_transform(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                            const float* i_ref, float floor_, DtLayout& L, cudaStream_t st, bool raw) {
  fkk_status s;
  L.n = n;
  L.m = m;
  L.np = ((n + 63) / 64) * 64;
  if (L.np == 0) L.np = 64;
  L.mg = ((m + 255) / 256) * 256;
  size_t dt_elems = (size_t)L.mg * (size_t)L.np;
  L.dt_hi = (__nv_bfloat16*)workspace(ctx, "dt_hi", dt_elems * 2, &s);
  if (!L.dt_hi) return s;
  L.dt_lo = (__nv_bfloat16*)workspace(ctx, "dt_lo", dt_elems * 2, &s);
  if (!L.dt_lo) return s;
  L.c = (float*)workspace(ctx, "shift_c", (size_t)m * 4, &s);
  if (!L.c) return s;
  L.sum_d = (double*)workspace(ctx, "sum_d", (size_t)m * 8, &s);
  if (!L.sum_d) return s;
  L.sum_i = (double*)workspace(ctx, "sum_i", (size_t)m * 8, &s);
  if (!L.sum_i) return s;
  L.sum_d2 = (double*)workspace(ctx, "sum_d2", (size_t)m * 8, &s);
  if (!L.sum_d2) return s;
  const int ctiles = L.mg / 64;
  const int64_t nrt = L.np / 64;
  int64_t grows = (int64_t)ctx->sm_count * 8 / ctiles;
  if (grows < 1) grows = 1;
  if (grows > nrt) grows = nrt;
  double* part_d = (double*)workspace(ctx, "part_d", (size_t)grows * m * 8, &s);
  if (!part_d) return s;
  double* part_i = (double*)workspace(ctx, "part_i", (size_t)grows * m * 8, &s);
  if (!part_i) return s;
  double* part_d2 = (double*)workspace(ctx, "part_d2", (size_t)grows * m * 8, &s);
  if (!part_d2) return s;
  FKK_COUNT_LAUNCH(); shift_kernel<<<(m + 127) / 128, 128, 0, st>>>(i_cars, n, m, ld, i_ref, floor_, L.c, raw ? 1 : 0);
  TransformArgs a{i_cars, n, m, ld, i_ref, floor_, L.c, L.np, L.dt_hi, L.dt_lo, part_d, part_i, part_d2, ctx->d_status};
  FKK_COUNT_LAUNCH();
  if (raw)
    transform_kernel<true><<<dim3((unsigned)grows, ctiles), 256, 0, st>>>(a);
  else
    transform_kernel<false><<<dim3((unsigned)grows, ctiles), 256, 0, st>>>(a);
  FKK_COUNT_LAUNCH();
  colsum_reduce_kernel<<<(m + 127) / 128, 128, 0, st>>>(part_d, part_i, part_d2, (int)grows, m, L.sum_d, L.sum_i,
                                                        L.sum_d2);
  return cuda_check(ctx, cudaGetLastError(), "transform launch");
}

}  // namespace fkk
