// Context, error and workspace management for the C ABI (include/fkk.h).
#include <cstring>
#include <new>

#include "fkk_internal.h"

namespace fkk {

std::atomic<unsigned long long> g_launches{0};

fkk_status fail(fkk_ctx* ctx, fkk_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

fkk_status cuda_check(fkk_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FKK_OK;
  return fail(ctx, FKK_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

fkk_status side_stream(fkk_ctx* ctx, cudaStream_t* out) {
  if (!ctx->aux) {
    FKK_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    FKK_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    FKK_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  }
  *out = ctx->aux;
  return FKK_OK;
}
bool is_host_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of a pointer the runtime does not know
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

fkk_status bind(fkk_ctx* ctx) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  return cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
}

void* workspace(fkk_ctx* ctx, const char* name, size_t bytes, fkk_status* st) {
  *st = FKK_OK;
  if (bytes == 0) bytes = 256;
  auto& b = ctx->ws[name];
  if (b.bytes >= bytes) return b.ptr;
  size_t grow = bytes - b.bytes;
  if (ctx->budget && ctx->used + grow > ctx->budget) {
    *st = fail(ctx, FKK_ERR_BUDGET, "workspace '%s' needs %zu bytes; budget %zu, in use %zu", name,
               bytes, ctx->budget, ctx->used);
    return nullptr;
  }
  if (b.ptr) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      *st = cuda_check(ctx, e, "cudaDeviceSynchronize (workspace grow)");
      return nullptr;
    }
    cudaFree(b.ptr);
    ctx->used -= b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    *st = cuda_check(ctx, e, "cudaMalloc (workspace)");
    return nullptr;
  }
  b.ptr = p;
  b.bytes = bytes;
  ctx->used += bytes;
  return p;
}

}  // namespace fkk

using namespace fkk;

extern "C" {

const char* fkk_strerror(fkk_status s) {
  switch (s) {
    case FKK_OK: return "FKK_OK";
    case FKK_ERR_INVALID_ARG: return "FKK_ERR_INVALID_ARG";
    case FKK_ERR_BUDGET: return "FKK_ERR_BUDGET";
    case FKK_ERR_CUDA: return "FKK_ERR_CUDA";
    case FKK_ERR_TIMEOUT: return "FKK_ERR_TIMEOUT";
    case FKK_ERR_NOT_CONVERGED: return "FKK_ERR_NOT_CONVERGED";
    case FKK_ERR_BAD_FILE: return "FKK_ERR_BAD_FILE";
    case FKK_ERR_SHUTDOWN: return "FKK_ERR_SHUTDOWN";
    default: return "FKK_ERR_UNKNOWN";
  }
}

const char* fkk_version(void) { return "fkk 0.1 sm_103a"; }

uint64_t fkk_launch_count(void) { return g_launches.load(); }

fkk_status fkk_create(fkk_ctx** out, int32_t device, size_t hbm_budget_bytes) {
  if (!out) return FKK_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return FKK_ERR_INVALID_ARG;
  fkk_ctx* c = new (std::nothrow) fkk_ctx();
  if (!c) return FKK_ERR_INVALID_ARG;
  c->device = device;
  c->budget = hbm_budget_bytes;
  fkk_status s = bind(c);
  if (s == FKK_OK) s = cuda_check(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device), "sm count");
  if (s == FKK_OK) s = cuda_check(c, cudaMalloc(&c->d_status, kStatusWords * sizeof(long long)), "cudaMalloc(status)");
  if (s == FKK_OK) s = cuda_check(c, cudaMemset(c->d_status, 0, kStatusWords * sizeof(long long)), "cudaMemset(status)");
  if (s != FKK_OK) {
    if (c->d_status) cudaFree(c->d_status);
    delete c;
    return s;
  }
  *out = c;
  return FKK_OK;
}

fkk_status fkk_test_stall_next_eigensolve(fkk_ctx* ctx) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->stall_next_eig = 1;
  return FKK_OK;
}

fkk_status fkk_destroy(fkk_ctx* ctx) {
  if (!ctx) return FKK_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (int i = 0; i < 2; ++i) {
    if (ctx->lane_done[i]) cudaEventDestroy(ctx->lane_done[i]);
    if (ctx->lane_st[i]) cudaStreamDestroy(ctx->lane_st[i]);
    if (ctx->lane_ctx[i]) fkk_destroy(ctx->lane_ctx[i]);
  }
  if (ctx->lane_start) cudaEventDestroy(ctx->lane_start);
  for (auto& kv : ctx->ws)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->d_status) cudaFree(ctx->d_status);
  delete ctx;
  return FKK_OK;
}

const char* fkk_last_error(const fkk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

size_t fkk_workspace_bytes(const fkk_ctx* ctx) { return ctx ? ctx->used : 0; }

fkk_status fkk_sync_status(fkk_ctx* ctx, void* stream, int64_t* clamped) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  FKK_TRY(bind(ctx));
  cudaStream_t st = as_stream(stream);
  long long h[kStatusWords];
  FKK_CUDA(ctx, cudaStreamSynchronize(st));
  FKK_CUDA(ctx, cudaMemcpy(h, ctx->d_status, sizeof h, cudaMemcpyDeviceToHost));
  FKK_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof h));
  if (clamped) *clamped = h[1];
  return static_cast<fkk_status>(h[0]);
}

fkk_status fkk_set_timing(fkk_ctx* ctx, int32_t on) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (on < 0 || on > 2) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_set_timing: level %d not in 0..2", on);
  ctx->timing = on;
  ctx->ev_valid = false;
  return FKK_OK;
}

fkk_status fkk_stage_ms(fkk_ctx* ctx, float* ms, int32_t n) {
  if (!ctx || !ms || n < 1) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!ctx->ev_valid) return fail(ctx, FKK_ERR_INVALID_ARG, "no timed fit recorded");
  FKK_TRY(bind(ctx));
  FKK_CUDA(ctx, cudaEventSynchronize(ctx->ev[fkk_ctx::kStages]));
  for (int i = 0; i < n && i < fkk_ctx::kStages; ++i)
    FKK_CUDA(ctx, cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]));
  return FKK_OK;
}

fkk_status fkk_eig_phase_cycles(fkk_ctx* ctx, int64_t* cycles, int32_t n) {
  if (!ctx || !cycles || n < 1) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->ws.find("eig_phase_cycles");
  if (it == ctx->ws.end() || !it->second.ptr) return fail(ctx, FKK_ERR_INVALID_ARG, "no timed eigensolve recorded");
  FKK_TRY(bind(ctx));
  long long h[8];
  FKK_CUDA(ctx, cudaDeviceSynchronize());
  FKK_CUDA(ctx, cudaMemcpy(h, it->second.ptr, sizeof h, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n && i < 8; ++i) cycles[i] = h[i];
  return FKK_OK;
}

}  // extern "C"
