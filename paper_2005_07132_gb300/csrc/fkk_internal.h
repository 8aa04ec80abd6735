// Internal host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "../../include/fkk.h"

// Device status block, one per context (int64 words):
//   [0] first device-side error code (0 = none)
//   [1] number of ratios clamped to the floor
//   [2] spare / diagnostic
constexpr int kStatusWords = 4;

struct fkk_ctx {
  int device = 0;
  int sm_count = 0;
  size_t budget = 0;  // 0 = unlimited
  size_t used = 0;
  std::string last_error;
  long long* d_status = nullptr;
  struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
  };
  std::map<std::string, Buf> ws;
  std::recursive_mutex mu;
  // optional per-stage timing of the fit (CUDA events on the fit's stream)
  int timing = 0;  // 0 off, 1 stage events, 2 also the eigensolver phase clocks
  static constexpr int kStages = 6;  // transform, gram, eig, project, basis, recon
  cudaEvent_t ev[kStages + 1] = {};
  bool ev_valid = false;
  // side stream for work that overlaps the caller's stream inside one call
  // (forked and joined with the two events; created on first use)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // ring depth of the fused apply kernel (0 = the deepest that fits; the
  // serving autotuner sets it on its own context)
  int apply_stages = 0;
  // fkk_test_stall_next_eigensolve: the next eigensolve's first exchange
  // waits for a tag that is never published (its bounded wait runs out)
  int stall_next_eig = 0;
  // worker lanes of fkk_fit_many (own contexts and streams), created on first use
  fkk_ctx* lane_ctx[2] = {};
  cudaStream_t lane_st[2] = {};
  cudaEvent_t lane_done[2] = {};
  cudaEvent_t lane_start = nullptr;
};

namespace fkk {

// Number of kernels this library has launched (process-wide).
extern std::atomic<unsigned long long> g_launches;
#define FKK_COUNT_LAUNCH() (::fkk::g_launches.fetch_add(1, std::memory_order_relaxed))

// Record an error message on the context and return the status.
fkk_status fail(fkk_ctx* ctx, fkk_status s, const char* fmt, ...);

// Map a CUDA error to FKK_ERR_CUDA with a message (FKK_OK if no error).
fkk_status cuda_check(fkk_ctx* ctx, cudaError_t e, const char* what);

// Named grow-only workspace buffer.  Returns nullptr and records an error
// (FKK_ERR_BUDGET or FKK_ERR_CUDA in *st) if it cannot be provided.  Growing
// synchronises the device first, so buffers in use by queued work are safe.
void* workspace(fkk_ctx* ctx, const char* name, size_t bytes, fkk_status* st);

// Make the context's device current for this host thread.
fkk_status bind(fkk_ctx* ctx);

// The context's side stream (created on first use, with its fork / join events).
fkk_status side_stream(fkk_ctx* ctx, cudaStream_t* out);

// Whether p points to host memory (pinned or pageable) rather than device or
// managed memory.
bool is_host_ptr(const void* p);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Record the boundary event `i` of the fit's stages when timing is on.
inline void stage_mark(fkk_ctx* ctx, int i, cudaStream_t st) {
  if (!ctx->timing) return;
  if (!ctx->ev[i]) cudaEventCreate(&ctx->ev[i]);
  cudaEventRecord(ctx->ev[i], st);
  if (i == fkk_ctx::kStages) ctx->ev_valid = true;
}

inline int next_pow2(int64_t x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace fkk

#define FKK_TRY(expr)                 \
  do {                                \
    fkk_status _s = (expr);           \
    if (_s != FKK_OK) return _s;      \
  } while (0)

#define FKK_CUDA(ctx, expr) FKK_TRY(::fkk::cuda_check((ctx), (expr), #expr))
