// fkk_reconstruct_noalloc: the tensor-core reconstruction (Eq. fKKEC) with
// its packed operands in fixed, statically sized device arrays, for callers
// that must not allocate device memory after start-up (a serving process
// with a fixed HBM footprint, or a loop that cannot afford the implicit
// device synchronisation of cudaMalloc / cudaFree).  The regular entry point
// packs into the context's grow-only workspace instead.  Not part of the
// paper's method.
//
// Scratch: bf16 hi / lo copies of P (up to 16384 rows x K = 128) and of the
// interleaved amplitude / phase coefficients (up to 2 x 2048 rows x 128),
// 10 MiB in all per device.  The packing kernels rewrite every element the
// GEMM reads, zero padding included, so nothing has to be cleared.  The
// arrays are process-wide: calls that overlap on the device race on them.
#include <cuda_bf16.h>

#include <mutex>

#include "../../include/fkk.h"
#include "fit.h"
#include "fkk_internal.h"

namespace fkk {
namespace {

constexpr int64_t kMaxRows = FKK_NOALLOC_MAX_SPECTRA;      // multiple of the 128-row tile
constexpr int64_t kMaxCRows = 2 * FKK_NOALLOC_MAX_CHANNELS;  // multiple of the 256-column tile
constexpr int64_t kMaxKp = 128;
static_assert(kMaxRows % 128 == 0 && kMaxCRows % 256 == 0, "scratch must hold whole tiles");

static __device__ __align__(256) __nv_bfloat16 g_p_hi[kMaxRows * kMaxKp];
static __device__ __align__(256) __nv_bfloat16 g_p_lo[kMaxRows * kMaxKp];
static __device__ __align__(256) __nv_bfloat16 g_c_hi[kMaxCRows * kMaxKp];
static __device__ __align__(256) __nv_bfloat16 g_c_lo[kMaxCRows * kMaxKp];

struct Scratch {
  bool ready = false;
  void* p_hi = nullptr;
  void* p_lo = nullptr;
  void* c_hi = nullptr;
  void* c_lo = nullptr;
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
Scratch g_scratch[kMaxDevices];

// Addresses of the static arrays on ctx's device, looked up once per device.
fkk_status scratch_for(fkk_ctx* ctx, Scratch* out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct_noalloc: device %d out of range", ctx->device);
  std::lock_guard<std::mutex> lk(g_mu);
  Scratch& s = g_scratch[ctx->device];
  if (!s.ready) {
    Scratch t;
    FKK_CUDA(ctx, cudaGetSymbolAddress(&t.p_hi, g_p_hi));
    FKK_CUDA(ctx, cudaGetSymbolAddress(&t.p_lo, g_p_lo));
    FKK_CUDA(ctx, cudaGetSymbolAddress(&t.c_hi, g_c_hi));
    FKK_CUDA(ctx, cudaGetSymbolAddress(&t.c_lo, g_c_lo));
    t.ready = true;
    s = t;
  }
  *out = s;
  return FKK_OK;
}

}  // namespace
}  // namespace fkk

using namespace fkk;

extern "C" fkk_status fkk_reconstruct_noalloc(fkk_ctx* ctx, const float* p, int64_t n, int32_t k, int32_t m,
                                              const double* c_amp, const double* c_ph, float* im, float* re,
                                              int64_t ld_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (n < 0 || n > kMaxRows)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct_noalloc: n_spectra %lld outside [0, %d]", (long long)n,
                FKK_NOALLOC_MAX_SPECTRA);
  if (m < 1 || m > FKK_NOALLOC_MAX_CHANNELS)
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct_noalloc: m %d outside [1, %d]", m,
                FKK_NOALLOC_MAX_CHANNELS);
  if (k < 1 || k > 80) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct_noalloc: k %d outside [1, 80]", k);
  if (ld_out < m) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct_noalloc: ld_out %lld < m", (long long)ld_out);
  FKK_TRY(bind(ctx));
  Scratch s;
  FKK_TRY(scratch_for(ctx, &s));
  if (n == 0) return FKK_OK;
  if (!p || !c_amp || !c_ph || !im) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_reconstruct_noalloc: null pointer");
  return launch_reconstruct_tc_scratch(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, as_stream(stream), s.p_hi,
                                       s.p_lo, s.c_hi, s.c_lo);
}
