// Serving of a trained basis (Sec. 2.6, ML:fKK-EC: new spectra are
// projected on the frozen basis, Eq. ML_Unew, and reconstructed with the
// cached coefficients, Eq. fKKEC), and the noise-model helper of Sec. 2.2.
//
// Continuous batching over kSlots in-flight batch slots.  Each slot owns a
// CUDA stream and device staging (input and output) of `cap` spectra, sized
// from the context's HBM budget; the staging is the admission resource.
// A dispatcher thread takes queued requests in submission order into the
// first free slot: consecutive host tiles are gathered into one batch while
// they fit the slot (one fused apply launch for all of them), a device tile
// runs alone in place.  The slot's work -- host-to-device copies, the apply
// (replayed from a CUDA graph captured per 1,024-row bucket), device-to-host
// copies -- is enqueued on its stream and the dispatcher moves on, so the
// copies of one batch overlap the kernel of another.  A host function at the
// end of each slot's stream marks the batch complete, records latency and
// frees the slot.  A request that finds no free slot waits in the queue
// (admission deferred); a host tile larger than a slot can never be staged
// and is refused with FKK_ERR_BUDGET.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "basis_internal.h"
#include "fit.h"

using Clock = std::chrono::steady_clock;

namespace fkk {
namespace {

constexpr int kSlots = 3;
constexpr int64_t kBucket = 1024;      // graph row bucket
constexpr int kLogRows = 1024;         // batch log ring

__global__ void noise_f_kernel(const float* __restrict__ mean, int m, double alpha, double sigma_g,
                               double* __restrict__ f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double mu = (double)mean[j];
  f[j] = 2.0 * mu / sqrt(alpha * mu + sigma_g * sigma_g);
}

__global__ void fill_kernel(float* __restrict__ x, int64_t n, float v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

}  // namespace
}  // namespace fkk

using namespace fkk;

struct fkk_req_state {
  const float* tile = nullptr;
  int64_t n = 0;
  bool host = false;
  float* out = nullptr;
  Clock::time_point t_submit;
  int state = 0;  // 0 queued, 1 running, 2 done
  fkk_status status = FKK_OK;
};

struct serve_slot {
  int index = 0;
  cudaStream_t stream = nullptr;
  float* d_in = nullptr;   // cap x m
  float* d_out = nullptr;  // cap x m
  bool busy = false;
  std::vector<uint64_t> batch;
  int log_row = -1;
  std::map<int64_t, cudaGraphExec_t> graphs;  // bucket rows -> captured apply
};

struct serve_log_row {
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  int slot = -1, nreq = 0;
  int64_t spectra = 0;
  bool done = false;
};

struct fkk_server {
  fkk_ctx* ctx = nullptr;  // the server's own context (workspace isolated from the caller's)
  const fkk_basis* basis = nullptr;
  int m = 0;
  int device = 0;
  int64_t cap = 0;  // spectra per slot
  bool use_graphs = true;
  serve_slot slots[kSlots];
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stopping = false;
  int waiters = 0;
  int busy = 0;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, fkk_req_state> reqs;
  uint64_t next_id = 1;
  // batch log (device events) and latency statistics
  cudaEvent_t origin = nullptr;
  serve_log_row log[kLogRows];
  int64_t log_next = 0;
  std::vector<double> lat_ms;  // ring of the last kLat latencies
  size_t lat_pos = 0;
  double spectra_done = 0.0;
  bool have_first = false;
  Clock::time_point t_first, t_last;
  static constexpr size_t kLat = 1 << 14;
};

namespace {

struct done_msg {
  fkk_server* S;
  int slot;
};

// Host function at the end of a slot's stream: the batch is complete.  No
// CUDA calls here.
void CUDART_CB slot_done(void* arg) {
  done_msg* d = static_cast<done_msg*>(arg);
  fkk_server* S = d->S;
  const Clock::time_point now = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    serve_slot& sl = S->slots[d->slot];
    for (uint64_t id : sl.batch) {
      auto it = S->reqs.find(id);
      if (it == S->reqs.end()) continue;
      fkk_req_state& r = it->second;
      if (r.state != 2) {
        r.state = 2;
        const double ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
        if (S->lat_ms.size() < fkk_server::kLat) S->lat_ms.push_back(ms);
        else S->lat_ms[S->lat_pos++ % fkk_server::kLat] = ms;
        if (r.status == FKK_OK) S->spectra_done += (double)r.n;
      }
    }
    if (sl.log_row >= 0) S->log[sl.log_row].done = true;
    sl.batch.clear();
    sl.busy = false;
    --S->busy;
    S->t_last = now;
  }
  S->cv_done.notify_all();
  S->cv_work.notify_all();
  delete d;
}

// Captures the fused apply over `bucket` rows of the slot's staging into a
// graph; false (and graphs off for good) if capture is unavailable.
bool capture_bucket(fkk_server* S, serve_slot& sl, int64_t bucket) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  bool ok = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  fkk_status s = FKK_OK;
  if (ok) s = fkk_apply(S->ctx, S->basis, sl.d_in, bucket, S->m, sl.d_out, nullptr, S->m, sl.stream);
  if (ok) ok = cudaStreamEndCapture(sl.stream, &g) == cudaSuccess && s == FKK_OK;
  if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    S->use_graphs = false;
    return false;
  }
  sl.graphs.emplace(bucket, ge);
  return true;
}

int64_t bucket_of(const fkk_server* S, int64_t rows) {
  const int64_t b = ((rows + kBucket - 1) / kBucket) * kBucket;
  return b > S->cap ? S->cap : b;
}

// The fused apply over `rows` rows of the slot's staging, replayed from the
// graph of its 1,024-row bucket (all captured by fkk_serve_start).
fkk_status slot_apply(fkk_server* S, serve_slot& sl, int64_t rows) {
  const int m = S->m;
  const int64_t bucket = bucket_of(S, rows);
  if (S->use_graphs) {
    auto it = sl.graphs.find(bucket);
    if (it == sl.graphs.end() && capture_bucket(S, sl, bucket)) it = sl.graphs.find(bucket);
    if (it != sl.graphs.end())
      return cudaGraphLaunch(it->second, sl.stream) == cudaSuccess ? FKK_OK : FKK_ERR_CUDA;
  }
  return fkk_apply(S->ctx, S->basis, sl.d_in, rows, m, sl.d_out, nullptr, m, sl.stream);
}

// Enqueue one batch on its slot's stream (called without the lock).
fkk_status issue_batch(fkk_server* S, serve_slot& sl, const std::vector<fkk_req_state*>& batch) {
  const int m = S->m;
  const size_t row = (size_t)m * sizeof(float);
  cudaStream_t st = sl.stream;
  if (batch.size() == 1 && !batch[0]->host) {  // a device tile, in place
    fkk_req_state* r = batch[0];
    return fkk_apply(S->ctx, S->basis, r->tile, r->n, m, r->out, nullptr, m, st);
  }
  int64_t off = 0;
  for (fkk_req_state* r : batch) {
    if (cudaMemcpyAsync(sl.d_in + off * m, r->tile, r->n * row,
                        r->host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FKK_ERR_CUDA;
    off += r->n;
  }
  FKK_TRY(slot_apply(S, sl, off));
  off = 0;
  for (fkk_req_state* r : batch) {
    if (cudaMemcpyAsync(r->out, sl.d_out + off * m, r->n * row,
                        r->host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FKK_ERR_CUDA;
    off += r->n;
  }
  return FKK_OK;
}

void worker_loop(fkk_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_work.wait(lk, [&] { return S->stopping || (!S->queue.empty() && S->busy < kSlots); });
    if (S->stopping && S->queue.empty()) break;
    if (S->queue.empty() || S->busy >= kSlots) continue;
    serve_slot* sl = nullptr;
    for (auto& x : S->slots)
      if (!x.busy) {
        sl = &x;
        break;
      }
    // continuous batching: queued requests in order while they fit the slot
    std::vector<fkk_req_state*> batch;
    int64_t total = 0;
    while (!S->queue.empty()) {
      const uint64_t id = S->queue.front();
      fkk_req_state* r = &S->reqs[id];
      if (!r->host) {
        if (!batch.empty()) break;
      } else if (!batch.empty() && (!batch.back()->host || total + r->n > S->cap)) {
        break;
      }
      S->queue.pop_front();
      r->state = 1;
      batch.push_back(r);
      sl->batch.push_back(id);
      total += r->n;
      if (!r->host) break;
    }
    sl->busy = true;
    ++S->busy;
    const int lr = (int)(S->log_next++ % kLogRows);
    serve_log_row& L = S->log[lr];
    L.slot = sl->index;
    L.nreq = (int)batch.size();
    L.spectra = total;
    L.done = false;
    sl->log_row = lr;
    lk.unlock();
    fkk_status s = cudaEventRecord(L.t0, sl->stream) == cudaSuccess ? FKK_OK : FKK_ERR_CUDA;
    if (s == FKK_OK) s = issue_batch(S, *sl, batch);
    if (s == FKK_OK && cudaEventRecord(L.t1, sl->stream) != cudaSuccess) s = FKK_ERR_CUDA;
    done_msg* msg = new done_msg{S, sl->index};
    if (s != FKK_OK) {
      for (fkk_req_state* r : batch) r->status = s;
    }
    if (cudaLaunchHostFunc(sl->stream, slot_done, msg) != cudaSuccess) {
      // the stream is unusable: complete the batch here
      cudaStreamSynchronize(sl->stream);
      for (fkk_req_state* r : batch) r->status = FKK_ERR_CUDA;
      slot_done(msg);
    }
    lk.lock();
  }
  // stopping: let every slot's work finish before the streams go away
  S->cv_done.wait(lk, [&] { return S->busy == 0; });
}

// Spectra per slot: the tune cache's max_batch when present, else 65,536;
// either way no more than the budget leaves room for (input and output
// staging of every slot), a multiple of 128.
int64_t pick_cap(fkk_ctx* ctx, int m, int64_t max_batch) {
  int64_t cap = max_batch;
  if (ctx->budget) {
    const size_t room = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
    const int64_t fit = (int64_t)(room / ((size_t)kSlots * 2 * m * sizeof(float)));
    cap = std::min(cap, fit);
  }
  return (cap / 128) * 128;
}

// Reads "max_batch=<n>" and "stages=<s>" lines; returns false if either is missing.
bool read_cache(const char* path, int64_t* max_batch, int* stages) {
  FILE* fp = std::fopen(path, "r");
  if (!fp) return false;
  char line[128];
  bool got_b = false, got_s = false;
  while (std::fgets(line, sizeof line, fp)) {
    long long v = 0;
    int sv = 0;
    if (std::sscanf(line, "max_batch=%lld", &v) == 1 && v >= 128 && v <= (1ll << 22)) {
      *max_batch = v;
      got_b = true;
    }
    if (std::sscanf(line, "stages=%d", &sv) == 1 && sv >= 0 && sv <= 4) {
      *stages = sv;
      got_s = true;
    }
  }
  std::fclose(fp);
  return got_b && got_s;
}

// Autotuner: times the fused apply on ratio-one spectra for each ring depth
// (2, 3, 4 where it fits shared memory) at the largest batch, then each
// batch size from 2,048 up with the best depth, and keeps the smallest batch
// within 10 % of the best throughput.
void calibrate(fkk_server* S, cudaStream_t st, int64_t* max_batch, int* stages) {
  fkk_ctx* ctx = S->ctx;
  const int m = S->m;
  FKK_COUNT_LAUNCH();
  fill_kernel<<<(unsigned)((S->cap * m + 255) / 256), 256, 0, st>>>(S->slots[0].d_in, S->cap * m, 1.0f);
  auto rate = [&](int64_t c) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fkk_apply(ctx, S->basis, S->slots[0].d_in, c, m, S->slots[0].d_out, nullptr, m, st);  // warm
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) fkk_apply(ctx, S->basis, S->slots[0].d_in, c, m, S->slots[0].d_out, nullptr, m, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return 3.0 * (double)c / (ms > 0.f ? ms : 1e-3f);
  };
  double best = 0.0;
  int best_s = 0;
  for (int s = 2; s <= 4; ++s) {
    ctx->apply_stages = s;
    const double r = rate(S->cap);
    if (r > best * 1.02) {
      best = r;
      best_s = s;
    }
  }
  ctx->apply_stages = best_s;
  *stages = best_s;
  std::vector<std::pair<int64_t, double>> rates;
  best = 0.0;
  for (int64_t c = 2048; c <= S->cap; c *= 2) {
    const double r = rate(c);
    rates.emplace_back(c, r);
    best = std::max(best, r);
  }
  *max_batch = S->cap;
  for (auto& r : rates)
    if (r.second >= 0.9 * best) {
      *max_batch = r.first;
      break;
    }
}

void free_slots(fkk_server* S) {
  for (auto& sl : S->slots) {
    for (auto& g : sl.graphs) cudaGraphExecDestroy(g.second);
    sl.graphs.clear();
    if (sl.stream) cudaStreamDestroy(sl.stream);
    sl.stream = nullptr;
  }
  for (auto& L : S->log) {
    if (L.t0) cudaEventDestroy(L.t0);
    if (L.t1) cudaEventDestroy(L.t1);
    L.t0 = L.t1 = nullptr;
  }
  if (S->origin) cudaEventDestroy(S->origin);
  S->origin = nullptr;
}

}  // namespace

extern "C" {

fkk_status fkk_noise_scale(fkk_ctx* ctx, const float* mean_spectrum, int32_t n_channels, double alpha,
                           double sigma_g, double* f_out, void* stream) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!mean_spectrum || !f_out || n_channels < 1 || !(alpha >= 0.0) || !(sigma_g >= 0.0) ||
      (alpha == 0.0 && sigma_g == 0.0))
    return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_noise_scale: bad arguments");
  FKK_TRY(bind(ctx));
  FKK_COUNT_LAUNCH();
  noise_f_kernel<<<(n_channels + 127) / 128, 128, 0, as_stream(stream)>>>(mean_spectrum, n_channels, alpha, sigma_g,
                                                                          f_out);
  return cuda_check(ctx, cudaGetLastError(), "fkk_noise_scale");
}

fkk_status fkk_serve_start(fkk_ctx* ctx, const fkk_basis* basis, const char* tune_cache, fkk_server** out) {
  if (!ctx) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!basis || !out) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_serve_start: null argument");
  int32_t m = 0;
  FKK_TRY(fkk_basis_info(basis, &m, nullptr, nullptr, nullptr));
  FKK_TRY(bind(ctx));
  fkk_server* S = new (std::nothrow) fkk_server();
  if (!S) return fail(ctx, FKK_ERR_INVALID_ARG, "fkk_serve_start: out of host memory");
  fkk_ctx* own = nullptr;
  if (fkk_status e = fkk_create(&own, ctx->device, ctx->budget)) {
    delete S;
    return fail(ctx, e, "fkk_serve_start: server context");
  }
  S->ctx = own;
  S->basis = basis;
  S->m = m;
  S->device = ctx->device;
  auto cleanup = [&](fkk_status e) {
    free_slots(S);
    if (e && own->last_error.size()) ctx->last_error = own->last_error;
    fkk_destroy(own);
    delete S;
    return e;
  };
  int64_t max_batch = 65536;
  int stages = 0;
  const bool cached = tune_cache && read_cache(tune_cache, &max_batch, &stages);
  own->apply_stages = stages;
  // the basis' packed operands (the apply must not synchronise inside a graph capture)
  fkk_status s = apply_pack(own, basis, nullptr);
  if (s) return cleanup(s);
  S->cap = pick_cap(own, m, max_batch);
  if (S->cap < 128)
    return cleanup(fail(ctx, FKK_ERR_BUDGET, "fkk_serve_start: the HBM budget leaves no room for %d staging slots",
                        kSlots));
  for (int i = 0; i < kSlots; ++i) {
    serve_slot& sl = S->slots[i];
    sl.index = i;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(ctx, FKK_ERR_CUDA, "fkk_serve_start: stream"));
    char name[64];
    std::snprintf(name, sizeof name, "serve_in_%d", i);
    sl.d_in = (float*)workspace(own, name, (size_t)S->cap * m * sizeof(float), &s);
    if (!sl.d_in) return cleanup(s);
    std::snprintf(name, sizeof name, "serve_out_%d", i);
    sl.d_out = (float*)workspace(own, name, (size_t)S->cap * m * sizeof(float), &s);
    if (!sl.d_out) return cleanup(s);
    cudaMemsetAsync(sl.d_in, 0, (size_t)S->cap * m * sizeof(float), sl.stream);
  }
  for (auto& L : S->log)
    if (cudaEventCreate(&L.t0) != cudaSuccess || cudaEventCreate(&L.t1) != cudaSuccess)
      return cleanup(fail(ctx, FKK_ERR_CUDA, "fkk_serve_start: events"));
  if (tune_cache && !cached) {
    calibrate(S, S->slots[0].stream, &max_batch, &stages);
    S->cap = std::min<int64_t>(S->cap, (max_batch / 128) * 128);
    if (FILE* fp = std::fopen(tune_cache, "w")) {
      std::fprintf(fp, "max_batch=%lld\nstages=%d\n", (long long)S->cap, stages);
      std::fclose(fp);
    }
  }
  // every bucket's graph on every slot up front, so that no request pays for
  // a capture and an instantiation
  for (auto& sl : S->slots) {
    cudaStreamSynchronize(sl.stream);
    for (int64_t b = kBucket; S->use_graphs; b += kBucket) {
      const int64_t bucket = bucket_of(S, b);
      if (!sl.graphs.count(bucket)) capture_bucket(S, sl, bucket);
      if (bucket >= S->cap) break;
    }
  }
  for (auto& sl : S->slots) cudaStreamSynchronize(sl.stream);
  if (cudaEventCreate(&S->origin) != cudaSuccess || cudaEventRecord(S->origin, S->slots[0].stream) != cudaSuccess ||
      cudaStreamSynchronize(S->slots[0].stream) != cudaSuccess)
    return cleanup(fail(ctx, FKK_ERR_CUDA, "fkk_serve_start: origin event"));
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return FKK_OK;
}

fkk_status fkk_serve_submit(fkk_server* S, const float* tile, int64_t n_spectra, int32_t tile_on_host,
                            float* im_out, fkk_req* out_id) {
  if (!S || !tile || !im_out || !out_id || n_spectra < 1) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) return FKK_ERR_SHUTDOWN;
  if (tile_on_host && n_spectra > S->cap) return FKK_ERR_BUDGET;  // can never be staged
  const uint64_t id = S->next_id++;
  fkk_req_state& r = S->reqs[id];
  r.tile = tile;
  r.n = n_spectra;
  r.host = tile_on_host != 0;
  r.out = im_out;
  r.t_submit = Clock::now();
  if (!S->have_first) {
    S->have_first = true;
    S->t_first = r.t_submit;
  }
  S->queue.push_back(id);
  *out_id = id;
  S->cv_work.notify_one();
  return FKK_OK;
}

fkk_status fkk_serve_wait(fkk_server* S, fkk_req id, int32_t timeout_ms) {
  if (!S) return FKK_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return FKK_ERR_INVALID_ARG;
  ++S->waiters;
  auto done = [&] {
    auto f = S->reqs.find(id);
    return f == S->reqs.end() || f->second.state == 2;  // gone: another waiter took it
  };
  bool ok;
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, done);
    ok = true;
  } else {
    ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  }
  --S->waiters;
  S->cv_done.notify_all();  // stop may be waiting for the waiter count
  if (!ok) return FKK_ERR_TIMEOUT;
  auto f = S->reqs.find(id);
  if (f == S->reqs.end()) return FKK_ERR_INVALID_ARG;
  const fkk_status st = f->second.status;
  S->reqs.erase(f);
  return st;
}

fkk_status fkk_serve_stats(fkk_server* S, double* p50_ms, double* p99_ms, double* spectra_per_s) {
  if (!S) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->lat_ms;
  double p50 = 0.0, p99 = 0.0;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
    p50 = q(0.50);
    p99 = q(0.99);
  }
  double rate = 0.0;
  if (S->have_first && S->spectra_done > 0.0) {
    const double sec = std::chrono::duration<double>(S->t_last - S->t_first).count();
    if (sec > 0.0) rate = S->spectra_done / sec;
  }
  if (p50_ms) *p50_ms = p50;
  if (p99_ms) *p99_ms = p99;
  if (spectra_per_s) *spectra_per_s = rate;
  return FKK_OK;
}

fkk_status fkk_serve_batch_log(fkk_server* S, double* out, int32_t max_rows, int32_t* n_rows) {
  if (!S || !n_rows || max_rows < 0 || (max_rows > 0 && !out)) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t first = std::max<int64_t>(0, S->log_next - kLogRows);
  int32_t n = 0;
  for (int64_t i = first; i < S->log_next && n < max_rows; ++i) {
    serve_log_row& L = S->log[i % kLogRows];
    if (!L.done) continue;
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, S->origin, L.t0) != cudaSuccess ||
        cudaEventElapsedTime(&b, S->origin, L.t1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    double* row = out + 5 * (size_t)n;
    row[0] = a;
    row[1] = b;
    row[2] = L.slot;
    row[3] = L.nreq;
    row[4] = (double)L.spectra;
    ++n;
  }
  *n_rows = n;
  return FKK_OK;
}

fkk_status fkk_serve_stop(fkk_server* S) {
  if (!S) return FKK_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    // queued requests are cancelled; batches already issued complete
    for (uint64_t id : S->queue) {
      fkk_req_state& r = S->reqs[id];
      r.state = 2;
      r.status = FKK_ERR_SHUTDOWN;
    }
    S->queue.clear();
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  {
    // threads blocked in fkk_serve_wait leave before the server goes away
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.notify_all();
    S->cv_done.wait(lk, [&] { return S->waiters == 0; });
  }
  for (auto& sl : S->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  free_slots(S);
  fkk_destroy(S->ctx);  // staging buffers and all workspace of the server
  delete S;
  return FKK_OK;
}

}  // extern "C"
