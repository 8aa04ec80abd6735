// Transform pass of the fit: d = 1/2 ln(max(I/I_ref, floor)) - c (or, in
// raw mode for the conventional workflow's SVD denoising, d = I - c), stored
// channel-major as two bf16 terms (D^T_hi, D^T_lo), plus per-channel sums of
// d and of I.  c is a per-channel shift (the mean log ratio of the first
// rows); it leaves A^T A unchanged in exact arithmetic,
//   sum_n a a^T = sum_n d d^T + s c^T + c s^T + N c c^T,  s = sum_n d,
// while shrinking the magnitudes the tensor-core Gram accumulates.
#include "common.cuh"
#include "df64.cuh"
#include "fit.h"
#include "tc.cuh"

namespace fkk {
namespace {

constexpr int kShiftRows = 256;

// c[j] = mean over the first min(n, 256) rows of d (before the shift): a
// block of 256 threads per 32 channels, each thread summing every 8th row of
// one channel, the 8 partial sums combined in a fixed order.
__global__ void __launch_bounds__(256) shift_kernel(const float* __restrict__ i_cars, int64_t n, int m, int64_t ld,
                                                    const float* __restrict__ i_ref, float floor_,
                                                    float* __restrict__ c, int raw) {
  __shared__ float part[8][33];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int rows = (int)(n < kShiftRows ? n : kShiftRows);
  float acc = 0.f;
  if (j < m) {
    const float rinv = raw ? 1.f : 1.f / i_ref[j];
    for (int t = g; t < rows; t += 8) {
      const float v = i_cars[(int64_t)t * ld + j];
      if (raw) {
        acc += v;
      } else {
        float x = v * rinv;
        x = (x >= floor_) ? x : floor_;
        acc += 0.5f * logf(x);
      }
    }
  }
  part[g][lane] = acc;
  __syncthreads();
  if (g == 0 && j < m) {
    float sum = 0.f;
    for (int q = 0; q < 8; ++q) sum += part[q][lane];
    c[j] = rows ? sum / (float)rows : 0.f;
  }
}

// log2 by the SFU (PTX lg2.approx.f32, relative error near 2^-22): far below
// the 2^-17 to which the bf16 hi + lo pair below represents d.
__device__ __forceinline__ float fast_log2(float x) {
  float y;
  asm("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Block = 256 threads, tile = 64 rows x 64 channels; blockIdx.x = channel
// tile (fastest, so that the tiles sharing rows run together and their
// DRAM bursts are read once); blockIdx.y walks row tiles rt = blockIdx.y,
// +gridDim.y, ...  Full tiles take a path without per-element bounds checks.
// kRaw: d = I - c (raw spectra; i_ref and the floor are not used).
template <bool kRaw>
__global__ void __launch_bounds__(256, 4) transform_kernel(TransformArgs p) {
  __shared__ float tile[64][65];
  __shared__ double red_d[4][64];
  __shared__ double red_d2[4][64];
  __shared__ double red_i[4][64];
  constexpr float kHalfLn2 = 0.34657359027997264f;  // d = 1/2 ln x = (ln 2 / 2) log2 x
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * 64;
  const int j = j0 + tx;
  const bool jvalid = j < p.m;
  const bool cfull = j0 + 64 <= p.m;
  const float rinv = (jvalid && !kRaw) ? 1.f / p.i_ref[j] : 1.f;
  const float cj = jvalid ? p.c[j] : 0.f;
  const float floor_ = p.floor_;
  const int64_t nrt = p.np / 64;
  const int64_t ld4 = 4 * p.ld;
  const int64_t ostep = 8 * p.np;
  double sum_d = 0.0, sum_i = 0.0, sum_d2 = 0.0;
  int clamped = 0;
  for (int64_t rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
    const int64_t n0 = rt * 64;
    const bool full = cfull && n0 + 64 <= p.n;
    const float* src = p.i_cars + (n0 + ty) * p.ld + j;
    float td = 0.f, ti = 0.f, td2 = 0.f;
    // all 16 loads of this thread in flight before any arithmetic
    float vals[16];
    if (full) {
#pragma unroll
      for (int u = 0; u < 16; ++u) vals[u] = __ldcs(src + u * ld4);
    } else {
#pragma unroll
      for (int u = 0; u < 16; ++u) vals[u] = (jvalid && n0 + ty + 4 * u < p.n) ? __ldcs(src + u * ld4) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const float v = vals[u];
      float d;
      if (kRaw) {
        d = v - cj;
      } else {
        const float x = v * rinv;
        const bool low = !(x >= floor_);  // also NaN
        d = fmaf(fast_log2(low ? floor_ : x), kHalfLn2, -cj);
        if (full || (jvalid && n0 + ty + 4 * u < p.n)) clamped += low;
      }
      if (!full && !(jvalid && n0 + ty + 4 * u < p.n)) d = 0.f;
      td += d;
      td2 = fmaf(d, d, td2);
      ti += v;  // 0 outside the cube
      tile[tx][ty + 4 * u] = d;
    }
    sum_d += td;
    sum_d2 += td2;
    sum_i += ti;
    __syncthreads();
    // transposed write: warp w handles channels w, w+8, ..., 32 lanes x 2 bf16;
    // hi = bf16(d), lo = bf16(d - hi), both rounded to nearest even
    __nv_bfloat16* oh = p.dt_hi + (int64_t)(j0 + w) * p.np + n0 + 2 * lane;
    __nv_bfloat16* ol = p.dt_lo + (int64_t)(j0 + w) * p.np + n0 + 2 * lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cc = w + 8 * q;
      const float a = tile[cc][2 * lane], b = tile[cc][2 * lane + 1];
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
      *reinterpret_cast<__nv_bfloat162*>(oh + q * ostep) = h;
      *reinterpret_cast<__nv_bfloat162*>(ol + q * ostep) = l;
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
    p.part_d[(int64_t)blockIdx.y * p.m + j] = sd;
    p.part_d2[(int64_t)blockIdx.y * p.m + j] = red_d2[0][tx] + red_d2[1][tx] + red_d2[2][tx] + red_d2[3][tx];
    p.part_i[(int64_t)blockIdx.y * p.m + j] = si;
  }
  for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
  if ((threadIdx.x & 31) == 0 && clamped)
    atomicAdd(reinterpret_cast<unsigned long long*>(p.status + 1), (unsigned long long)clamped);
}

// The same transform with the tiles moved by TMA (row stride a multiple of
// 16 bytes): a 3-stage ring of 64 x 64 fp32 input tiles (rows >= N and
// channels >= M read as 0), the d tile transposed through shared memory, and
// the bf16 hi / lo tiles staged in the input buffer just consumed and written
// by two TMA stores, so that no thread computes a global address per
// element.  Two tiles per CTA are in flight while it works on a third.
// Persistent CTAs: blockIdx.x = channel tile, blockIdx.y walks row tiles.
constexpr int kTtStages = 3;
constexpr int kTtBytesIn = 64 * 64 * 4;
constexpr size_t kTtSmem = 128 + kTtStages * kTtBytesIn + 64 * 65 * 4;

template <bool kRaw>
__global__ void __launch_bounds__(256, 3)
    transform_tma_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_hi,
                         const __grid_constant__ CUtensorMap tm_lo, TransformArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* ring = reinterpret_cast<float*>(sm);  // [stage][64 rows][64 ch]
  float(*tile)[65] = reinterpret_cast<float(*)[65]>(sm + kTtStages * kTtBytesIn);
  __shared__ double red_d[4][64];
  __shared__ double red_d2[4][64];
  __shared__ double red_i[4][64];
  __shared__ uint64_t full[kTtStages];
  __shared__ int fail_s;
  constexpr float kHalfLn2 = 0.34657359027997264f;
  const int tid = threadIdx.x;
  const int tx = tid & 63, ty = tid >> 6;
  const int w = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * 64;
  const int j = j0 + tx;
  const bool jvalid = j < p.m;
  const bool cfull = j0 + 64 <= p.m;
  const float rinv = (jvalid && !kRaw) ? 1.f / p.i_ref[j] : 1.f;
  const float cj = jvalid ? p.c[j] : 0.f;
  const float floor_ = p.floor_;
  const int64_t nrt = p.np / 64;
  const int64_t gstep = gridDim.y;
  // thread 0's bookkeeping (for the drain after a timeout): stages with a
  // load issued and not yet waited for, and the parity of each stage's next wait
  uint32_t pend = 0, wpar = 0;
  if (tid == 0) {
    tc::prefetch_tmap(&tm_in);
    tc::prefetch_tmap(&tm_hi);
    tc::prefetch_tmap(&tm_lo);
    for (int q = 0; q < kTtStages; ++q) tc::mbar_init(&full[q], 1);
    tc::fence_mbar_init();
    fail_s = 0;
    for (int q = 0; q < kTtStages - 1; ++q) {
      const int64_t r = blockIdx.y + q * gstep;
      if (r < nrt) {
        tc::mbar_arrive_expect_tx(&full[q], kTtBytesIn);
        tc::tma_load_2d(ring + q * 64 * 64, &tm_in, &full[q], j0, (int)(r * 64));
        pend |= 1u << q;
      }
    }
  }
  __syncthreads();
  // per-thread channel sums in double-word arithmetic on the fp32 pipe (the
  // fp64 pipe of this part would be a third busy with one add per tile)
  dw::df sum_d = dw::make(0.f), sum_i = dw::make(0.f), sum_d2 = dw::make(0.f);
  int clamped = 0;
  int it = 0;
  for (int64_t rt = blockIdx.y; rt < nrt; rt += gstep, ++it) {
    const int b = it % kTtStages;
    if (!tc::mbar_wait(&full[b], (it / kTtStages) & 1)) fail_s = 1;
    if (tid == 0) {
      pend &= ~(1u << b);
      wpar ^= 1u << b;
    }
    __syncthreads();
    if (fail_s) break;
    const int64_t n0 = rt * 64;
    const bool full_tile = cfull && n0 + 64 <= p.n;
    float* in = ring + b * 64 * 64;
    float td = 0.f, ti = 0.f, td2 = 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int r = ty + 4 * u;
      const float v = in[r * 64 + tx];
      const bool ok = full_tile || (jvalid && n0 + r < p.n);
      float d;
      if (kRaw) {
        d = v - cj;
      } else {
        const float x = v * rinv;
        const bool low = !(x >= floor_);  // also NaN
        d = fmaf(fast_log2(low ? floor_ : x), kHalfLn2, -cj);
        clamped += (ok && low) ? 1 : 0;
      }
      if (!ok) d = 0.f;
      td += d;
      td2 = fmaf(d, d, td2);
      ti += v;  // 0 outside the cube (TMA fill)
      tile[tx][r] = d;
    }
    sum_d = dw::add(sum_d, td);
    sum_d2 = dw::add(sum_d2, td2);
    sum_i = dw::add(sum_i, ti);
    const int64_t rn = rt + (kTtStages - 1) * gstep;
    if (tid == 0 && rn < nrt) {
      // stage (it + 2) % 3 held tile it - 1: consumed, and its stores (issued
      // a whole phase ago) must have read the hi / lo staged there
      const int q = (it + kTtStages - 1) % kTtStages;
      tc::bulk_wait_read0();
      tc::mbar_arrive_expect_tx(&full[q], kTtBytesIn);
      tc::tma_load_2d(ring + q * 64 * 64, &tm_in, &full[q], j0, (int)(rn * 64));
      pend |= 1u << q;
    }
    __syncthreads();
    // hi = bf16(d), lo = bf16(d - hi), both rounded to nearest even, staged in
    // the consumed input stage: word (cc, lane) holds rows 2 lane, 2 lane + 1
    uint32_t* out_hi = reinterpret_cast<uint32_t*>(in);
    uint32_t* out_lo = out_hi + 64 * 32;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cc = w + 8 * q;
      const float a = tile[cc][2 * lane], c2 = tile[cc][2 * lane + 1];
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, c2);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, c2 - hf.y);
      out_hi[cc * 32 + lane] = *reinterpret_cast<const uint32_t*>(&h);
      out_lo[cc * 32 + lane] = *reinterpret_cast<const uint32_t*>(&l);
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::tma_store_2d(&tm_hi, out_hi, (int)n0, j0);
      tc::tma_store_2d(&tm_lo, out_lo, (int)n0, j0);
      tc::bulk_commit();
    }
  }
  if (tid == 0) {
    tc::bulk_wait0();
    if (fail_s) {  // after a timed-out wait: let the loads still in flight land (bounded)
      for (int q = 0; q < kTtStages; ++q)
        if ((pend >> q) & 1u) tc::mbar_wait(&full[q], (wpar >> q) & 1u);
      record_error(p.status, kErrTimeout);
    }
  }
  red_d[ty][tx] = dw::to_double(sum_d);
  red_d2[ty][tx] = dw::to_double(sum_d2);
  red_i[ty][tx] = dw::to_double(sum_i);
  __syncthreads();
  if (ty == 0 && jvalid) {
    p.part_d[(int64_t)blockIdx.y * p.m + j] = red_d[0][tx] + red_d[1][tx] + red_d[2][tx] + red_d[3][tx];
    p.part_d2[(int64_t)blockIdx.y * p.m + j] = red_d2[0][tx] + red_d2[1][tx] + red_d2[2][tx] + red_d2[3][tx];
    p.part_i[(int64_t)blockIdx.y * p.m + j] = red_i[0][tx] + red_i[1][tx] + red_i[2][tx] + red_i[3][tx];
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
  const bool tma_ok = (ld % 4 == 0) && (reinterpret_cast<uintptr_t>(i_cars) % 16 == 0) && m >= 64 && n >= 64;
  int64_t grows = (int64_t)ctx->sm_count * (tma_ok ? 3 : 8) / ctiles;
  if (grows < 1) grows = 1;
  if (grows > nrt) grows = nrt;
  double* part_d = (double*)workspace(ctx, "part_d", (size_t)grows * m * 8, &s);
  if (!part_d) return s;
  double* part_i = (double*)workspace(ctx, "part_i", (size_t)grows * m * 8, &s);
  if (!part_i) return s;
  double* part_d2 = (double*)workspace(ctx, "part_d2", (size_t)grows * m * 8, &s);
  if (!part_d2) return s;
  FKK_COUNT_LAUNCH(); shift_kernel<<<(m + 31) / 32, 256, 0, st>>>(i_cars, n, m, ld, i_ref, floor_, L.c, raw ? 1 : 0);
  TransformArgs a{i_cars, n, m, ld, i_ref, floor_, L.c, L.np, L.dt_hi, L.dt_lo, part_d, part_i, part_d2, ctx->d_status};
  // TMA path: 16-byte aligned rows, at least one full tile each way
  if (tma_ok) {
    CUtensorMap tin, thi, tlo;
    FKK_TRY(make_tmap_2d(ctx, &tin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<float*>(i_cars), (uint64_t)m,
                         (uint64_t)n, (uint64_t)ld * 4, 64, 64, CU_TENSOR_MAP_SWIZZLE_NONE));
    FKK_TRY(make_tmap_2d(ctx, &thi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_hi, (uint64_t)L.np, (uint64_t)L.mg,
                         (uint64_t)L.np * 2, 64, 64, CU_TENSOR_MAP_SWIZZLE_NONE));
    FKK_TRY(make_tmap_2d(ctx, &tlo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_lo, (uint64_t)L.np, (uint64_t)L.mg,
                         (uint64_t)L.np * 2, 64, 64, CU_TENSOR_MAP_SWIZZLE_NONE));
    const void* fn = raw ? (const void*)transform_tma_kernel<true> : (const void*)transform_tma_kernel<false>;
    FKK_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTtSmem));
    FKK_COUNT_LAUNCH();
    if (raw)
      transform_tma_kernel<true><<<dim3(ctiles, (unsigned)grows), 256, kTtSmem, st>>>(tin, thi, tlo, a);
    else
      transform_tma_kernel<false><<<dim3(ctiles, (unsigned)grows), 256, kTtSmem, st>>>(tin, thi, tlo, a);
  } else {
    FKK_COUNT_LAUNCH();
    if (raw)
      transform_kernel<true><<<dim3(ctiles, (unsigned)grows), 256, 0, st>>>(a);
    else
      transform_kernel<false><<<dim3(ctiles, (unsigned)grows), 256, 0, st>>>(a);
  }
  FKK_COUNT_LAUNCH();
  colsum_reduce_kernel<<<(m + 127) / 128, 128, 0, st>>>(part_d, part_i, part_d2, (int)grows, m, L.sum_d, L.sum_i,
                                                        L.sum_d2);
  return cuda_check(ctx, cudaGetLastError(), "transform launch");
}

}  // namespace fkk
