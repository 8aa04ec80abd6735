// Many independent cubes fitted in one call (fKK-EC of Fig. 1(b) applied to
// each image on its own, Secs. 2.2-2.5): the jobs are dealt, largest first,
// to the less loaded of two worker lanes -- each a context of its own (its
// own workspace, kept on ctx for later calls) with its own stream -- so the
// stages of one cube overlap those of another where the device has room.
// Both lanes start after the work already queued on the caller's stream,
// the caller's stream waits for both at the end, and the lanes' device
// status (clamp counts, eigensolver failures) is folded into ctx's.
#include <algorithm>
#include <numeric>
#include <vector>

#include "fkk_internal.h"

namespace fkk {
namespace {

constexpr int kLanes = 2;

// ctx status += the lanes' (first error, clamp counts), lanes cleared
__global__ void fold_status_kernel(long long* __restrict__ dst, long long* __restrict__ a,
                                   long long* __restrict__ b) {
  if (threadIdx.x != 0) return;
  if (dst[0] == 0) dst[0] = a[0] ? a[0] : b[0];
  dst[1] += a[1] + b[1];
  a[0] = a[1] = b[0] = b[1] = 0;
}

fkk_status ensure_lanes(fkk_ctx* ctx) {
  for (int i = 0; i < kLanes; ++i) {
    if (!ctx->lane_ctx[i]) {
      fkk_status e = fkk_create(&ctx->lane_ctx[i], ctx->device, ctx->budget ? ctx->budget / kLanes : 0);
      if (e) return fail(ctx, e, "fkk_fit_many: worker context");
    }
    if (!ctx->lane_st[i] && cudaStreamCreateWithFlags(&ctx->lane_st[i], cudaStreamNonBlocking) != cudaSuccess)
      return fail(ctx, FKK_ERR_CUDA, "fkk_fit_many: worker stream");
    if (!ctx->lane_done[i] && cudaEventCreateWithFlags(&ctx->lane_done[i], cudaEventDisableTiming) != cudaSuccess)
      return fail(ctx, FKK_ERR_CUDA, "fkk_fit_many: worker event");
  }
  if (!ctx->lane_start && cudaEventCreateWithFlags(&ctx->lane_start, cudaEventDisableTiming) != cudaSuccess)
    return fail(ctx, FKK_ERR_CUDA, "fkk_fit_many: start event");
  return FKK_OK;
}

}  // namespace
}  // namespace fkk

using namespace fkk;

extern "C" fkk_status fkk_fit_many(fkk_ctx* ctx, int32_t n_jobs, const fkk_cube_job* jobs, fkk_basis** out_bases,
                                   void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !out_bases)))
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_fit_many: bad arguments");
  for (int32_t i = 0; i < n_jobs; ++i) out_bases[i] = nullptr;
  if (n_jobs == 0) return FKK_OK;
  FKK_TRY(bind(ctx));
  FKK_TRY(ensure_lanes(ctx));
  cudaStream_t st = as_stream(stream);
  auto bail = [&](fkk_status e) {
    for (int i = 0; i < kLanes; ++i) cudaStreamSynchronize(ctx->lane_st[i]);
    for (int32_t i = 0; i < n_jobs; ++i) {
      fkk_basis_free(out_bases[i]);
      out_bases[i] = nullptr;
    }
    return e;
  };
  FKK_CUDA(ctx, cudaEventRecord(ctx->lane_start, st));
  for (int i = 0; i < kLanes; ++i) FKK_CUDA(ctx, cudaStreamWaitEvent(ctx->lane_st[i], ctx->lane_start, 0));
  // largest first (by N M^2, the Gram's share), each to the lane with the least work so far
  std::vector<int32_t> order(n_jobs);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int32_t i) { return (double)jobs[i].n_spectra * jobs[i].n_channels * jobs[i].n_channels; };
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work(a) > work(b); });
  double load[kLanes] = {};
  for (int32_t i : order) {
    const fkk_cube_job& j = jobs[i];
    const int lane = load[1] < load[0] ? 1 : 0;
    load[lane] += work(i);
    fkk_status e = fkk_fit_basis(ctx->lane_ctx[lane], j.i_cars, j.n_spectra, j.n_channels, j.ld, j.i_ref,
                                 j.f_or_null, &j.params, &out_bases[i], j.im_out, j.re_out, j.ld_out,
                                 ctx->lane_st[lane]);
    if (e) {
      ctx->last_error = std::string("job ") + std::to_string(i) + ": " + ctx->lane_ctx[lane]->last_error;
      return bail(e);
    }
  }
  for (int i = 0; i < kLanes; ++i) {
    FKK_CUDA(ctx, cudaEventRecord(ctx->lane_done[i], ctx->lane_st[i]));
    FKK_CUDA(ctx, cudaStreamWaitEvent(st, ctx->lane_done[i], 0));
  }
  FKK_COUNT_LAUNCH();
  fold_status_kernel<<<1, 32, 0, st>>>(ctx->d_status, ctx->lane_ctx[0]->d_status, ctx->lane_ctx[1]->d_status);
  return cuda_check(ctx, cudaGetLastError(), "fkk_fit_many");
}
