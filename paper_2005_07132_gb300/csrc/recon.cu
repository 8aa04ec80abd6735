// Reconstruction, Eq. fKKEC with U S = P:
//   Im{K}[n, j] = exp((P C_amp)[n, j]) sin((P C_ph)[n, j])
//   Re{K}[n, j] = exp((P C_amp)[n, j]) cos((P C_ph)[n, j])
// One thread per output column j keeps its 2k coefficients in registers and
// walks a tile of rows whose P rows sit in shared memory.
#include "common.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr int kRowsPerBlock = 64;

template <int KC>
__global__ void __launch_bounds__(256) recon_kernel(const float* __restrict__ p, int64_t n, int k, int m,
                                                    const float* __restrict__ camp, const float* __restrict__ cph,
                                                    float* __restrict__ im, float* __restrict__ re,
                                                    int64_t ld_out) {
  __shared__ float ps[kRowsPerBlock][KC];
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  const int64_t rem = n - r0;
  const int rows = rem < kRowsPerBlock ? (int)rem : kRowsPerBlock;
  for (int t = threadIdx.x; t < kRowsPerBlock * KC; t += blockDim.x) {
    int r = t / KC, i = t % KC;
    ps[r][i] = (r < rows && i < k) ? p[(r0 + r) * k + i] : 0.f;
  }
  __syncthreads();
  if (j >= m) return;
  float ca[KC], cp[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) {
    ca[i] = (i < k) ? camp[(int64_t)i * m + j] : 0.f;
    cp[i] = (i < k) ? cph[(int64_t)i * m + j] : 0.f;
  }
  for (int r = 0; r < rows; ++r) {
    float x = 0.f, y = 0.f;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
      x = fmaf(ps[r][i], ca[i], x);
      y = fmaf(ps[r][i], cp[i], y);
    }
    float s, c;
    sincosf(y, &s, &c);
    const float e = expf(x);
    im[(r0 + r) * ld_out + j] = e * s;
    if (re) re[(r0 + r) * ld_out + j] = e * c;
  }
}

__global__ void to_f32_kernel(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

}  // namespace

fkk_status launch_reconstruct(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                              const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st) {
  fkk_status s;
  const size_t km = (size_t)k * m;
  float* ca = (float*)workspace(ctx, "rc_camp", km * 4, &s);
  if (!ca) return s;
  float* cp = (float*)workspace(ctx, "rc_cph", km * 4, &s);
  if (!cp) return s;
  FKK_COUNT_LAUNCH(); to_f32_kernel<<<(unsigned)((km + 255) / 256), 256, 0, st>>>(c_amp, (int64_t)km, ca);
  FKK_COUNT_LAUNCH(); to_f32_kernel<<<(unsigned)((km + 255) / 256), 256, 0, st>>>(c_ph, (int64_t)km, cp);
  dim3 grid((unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock), (m + 255) / 256);
  switch ((k + 7) / 8) {
#define FKK_RC(KB) \
  case KB: FKK_COUNT_LAUNCH(); recon_kernel<KB * 8><<<grid, 256, 0, st>>>(p, n, k, m, ca, cp, im, re, ld_out); break;
    FKK_RC(1) FKK_RC(2) FKK_RC(3) FKK_RC(4) FKK_RC(5) FKK_RC(6) FKK_RC(7) FKK_RC(8) FKK_RC(9) FKK_RC(10)
#undef FKK_RC
    default:
      return fail(ctx, FKK_ERR_INVALID_ARG, "k=%d outside 1..80", k);
  }
  return cuda_check(ctx, cudaGetLastError(), "recon launch");
}

}  // namespace fkk
