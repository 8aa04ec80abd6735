// Measured throughput of the double-word multiply-add that the eigensolver's
// Householder reduction is made of: the dot products and rank-2 updates of
// each column step are dw::add(acc, dw::mul(x, y)) on the fp32 pipe
// (df64.cuh: one FMA-based TwoProd product and one TwoSum-based sum, two
// flops in the 4/3 M^3 count of the reduction).  Every thread of a
// full-occupancy grid runs kRateChains independent chains
//   acc <- acc * y + x_c
// so the pipe, not a dependency, sets the rate; the chain values come back
// for a check against exact arithmetic on the host.
#include "common.cuh"
#include "df64.cuh"
#include "fkk_internal.h"

namespace fkk {
namespace {

constexpr int kRateThreads = 256;
constexpr int kRateChains = 8;

__global__ void __launch_bounds__(kRateThreads) dw_rate_kernel(dw::df y, dw::df x0, int iters,
                                                               double* __restrict__ chains,
                                                               double* __restrict__ sink) {
  dw::df x[kRateChains], acc[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) {
    x[c] = dw::ldexp(x0, -c);  // exact
    acc[c] = dw::make(0.f);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) acc[c] = dw::add(dw::mul(acc[c], y), x[c]);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += dw::to_double(acc[c]);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  sink[g] = s;  // every chain reaches memory, so none is removed
  if (g == 0)
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) chains[c] = dw::to_double(acc[c]);
}

}  // namespace
}  // namespace fkk

using namespace fkk;

extern "C" fkk_status fkk_dw_rate(fkk_ctx* ctx, int32_t iters, double* flops_per_s, double* chains_out,
                                  void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (iters < 1 || iters > (1 << 20) || (!flops_per_s && !chains_out))
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_dw_rate: bad arguments");
  FKK_TRY(bind(ctx));
  const cudaStream_t st = as_stream(stream);
  int per_sm = 0;
  FKK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dw_rate_kernel, kRateThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const int blocks = ctx->sm_count * per_sm;
  fkk_status s;
  double* chains = (double*)workspace(ctx, "dw_rate_chains", kRateChains * sizeof(double), &s);
  if (!chains) return s;
  double* sink = (double*)workspace(ctx, "dw_rate_sink", (size_t)blocks * kRateThreads * sizeof(double), &s);
  if (!sink) return s;
  // y = 1 - 2^-9 + 3 2^-33 and x0 = 0.1f + 2^-30: both words matter, the
  // fixed point x_c / (1 - y) is about 51 / 2^c
  const dw::df y{1.0f - 0.001953125f, 3.0f * 1.16415321826934814453125e-10f};
  const dw::df x0{0.1f, 9.31322574615478515625e-10f};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FKK_CUDA(ctx, cudaEventCreate(&e0));
  fkk_status out = cuda_check(ctx, cudaEventCreate(&e1), "fkk_dw_rate: event");
  if (out == FKK_OK) {
    FKK_COUNT_LAUNCH();  // warm-up: clocks up, code loaded
    dw_rate_kernel<<<blocks, kRateThreads, 0, st>>>(y, x0, iters < 256 ? iters : 256, chains, sink);
    cudaEventRecord(e0, st);
    FKK_COUNT_LAUNCH();
    dw_rate_kernel<<<blocks, kRateThreads, 0, st>>>(y, x0, iters, chains, sink);
    cudaEventRecord(e1, st);
    out = cuda_check(ctx, cudaGetLastError(), "dw_rate_kernel launch");
  }
  if (out == FKK_OK) out = cuda_check(ctx, cudaEventSynchronize(e1), "fkk_dw_rate: synchronise");
  float ms = 0.f;
  if (out == FKK_OK) out = cuda_check(ctx, cudaEventElapsedTime(&ms, e0, e1), "fkk_dw_rate: elapsed");
  if (out == FKK_OK && chains_out)
    out = cuda_check(ctx, cudaMemcpy(chains_out, chains, kRateChains * sizeof(double), cudaMemcpyDeviceToHost),
                     "fkk_dw_rate: copy");
  if (out == FKK_OK && flops_per_s)
    *flops_per_s = ms > 0.f ? 2.0 * (double)blocks * kRateThreads * kRateChains * (double)iters / (ms * 1e-3) : 0.0;
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return out;
}
