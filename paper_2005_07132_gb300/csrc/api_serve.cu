// Serving of a trained basis (Sec. 2.6, ML:fKK-EC: new spectra are
// projected on the frozen basis, Eq. ML_Unew, and reconstructed with the
// cached coefficients, Eq. fKKEC), and the noise-model helper of Sec. 2.2.
//
// A server owns one worker thread and one CUDA stream.  Requests (tiles of
// spectra, device-resident or in pinned host memory) queue in submission
// order; the worker takes as many queued tiles as fit its device staging
// buffers (continuous batching), gathers them into one contiguous block,
// runs fkk_apply once on the block and scatters the results back.  A tile
// larger than the staging buffers runs alone in chunks.  Latency is
// measured from submit to the moment the worker observes the batch's
// completion on the stream.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fkk_internal.h"

using Clock = std::chrono::steady_clock;

namespace fkk {
namespace {

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

struct fkk_server {
  fkk_ctx* ctx = nullptr;  // the server's own context (workspace isolated from the caller's)
  const fkk_basis* basis = nullptr;
  int m = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  float* d_in = nullptr;   // staging, cap x m
  float* d_out = nullptr;  // staging, cap x m
  int64_t cap = 0;         // spectra per batch
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stopping = false;
  int waiters = 0;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, fkk_req_state> reqs;
  uint64_t next_id = 1;
  // statistics
  std::vector<double> lat_ms;  // ring of the last kLat latencies
  size_t lat_pos = 0;
  double spectra_done = 0.0;
  bool have_first = false;
  Clock::time_point t_first, t_last;
  static constexpr size_t kLat = 1 << 14;
};

namespace {

// Runs one batch of requests (already marked running); returns its status.
fkk_status run_batch(fkk_server* S, const std::vector<std::pair<uint64_t, fkk_req_state*>>& batch) {
  const int m = S->m;
  const size_t row = (size_t)m * sizeof(float);
  cudaStream_t st = S->stream;
  if (batch.size() == 1 && !batch[0].second->host) {
    // a single device tile: apply in place
    fkk_req_state* r = batch[0].second;
    fkk_status s = fkk_apply(S->ctx, S->basis, r->tile, r->n, m, r->out, nullptr, m, st);
    if (s) return s;
    return cudaStreamSynchronize(st) == cudaSuccess ? FKK_OK : FKK_ERR_CUDA;
  }
  if (batch.size() == 1 && batch[0].second->n > S->cap) {
    // a host tile larger than the staging buffers: chunks
    fkk_req_state* r = batch[0].second;
    for (int64_t o = 0; o < r->n; o += S->cap) {
      const int64_t c = std::min<int64_t>(S->cap, r->n - o);
      if (cudaMemcpyAsync(S->d_in, r->tile + o * m, c * row, cudaMemcpyHostToDevice, st)) return FKK_ERR_CUDA;
      fkk_status s = fkk_apply(S->ctx, S->basis, S->d_in, c, m, S->d_out, nullptr, m, st);
      if (s) return s;
      if (cudaMemcpyAsync(r->out + o * m, S->d_out, c * row, cudaMemcpyDeviceToHost, st)) return FKK_ERR_CUDA;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? FKK_OK : FKK_ERR_CUDA;
  }
  int64_t off = 0;
  for (auto& e : batch) {
    fkk_req_state* r = e.second;
    if (cudaMemcpyAsync(S->d_in + off * m, r->tile, r->n * row,
                        r->host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st))
      return FKK_ERR_CUDA;
    off += r->n;
  }
  fkk_status s = fkk_apply(S->ctx, S->basis, S->d_in, off, m, S->d_out, nullptr, m, st);
  if (s) return s;
  off = 0;
  for (auto& e : batch) {
    fkk_req_state* r = e.second;
    if (cudaMemcpyAsync(r->out, S->d_out + off * m, r->n * row,
                        r->host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st))
      return FKK_ERR_CUDA;
    off += r->n;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? FKK_OK : FKK_ERR_CUDA;
}

void worker_loop(fkk_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_work.wait(lk, [&] { return S->stopping || !S->queue.empty(); });
    if (S->queue.empty()) break;  // stopping and drained
    // continuous batching: queued tiles in order while they fit
    std::vector<std::pair<uint64_t, fkk_req_state*>> batch;
    int64_t total = 0;
    while (!S->queue.empty()) {
      const uint64_t id = S->queue.front();
      fkk_req_state* r = &S->reqs[id];
      if (!batch.empty() && total + r->n > S->cap) break;
      S->queue.pop_front();
      r->state = 1;
      batch.emplace_back(id, r);
      total += r->n;
      if (total >= S->cap) break;
    }
    lk.unlock();
    const fkk_status s = run_batch(S, batch);
    const Clock::time_point now = Clock::now();
    lk.lock();
    for (auto& e : batch) {
      fkk_req_state* r = e.second;
      r->status = s;
      r->state = 2;
      const double ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
      if (S->lat_ms.size() < fkk_server::kLat) S->lat_ms.push_back(ms);
      else S->lat_ms[S->lat_pos++ % fkk_server::kLat] = ms;
      if (s == FKK_OK) S->spectra_done += (double)r->n;
    }
    S->t_last = now;
    S->cv_done.notify_all();
  }
}

// Staging size: the tune cache's max_batch when present, else the largest
// power of two up to 65,536 spectra that the budget leaves room for; with
// a cache path and no entry, a short calibration on synthetic tiles picks
// the smallest size within 10% of the best throughput and writes it.
int64_t pick_cap(fkk_ctx* ctx, const fkk_basis* basis, int m, const char* cache, bool* calibrate) {
  *calibrate = false;
  if (cache) {
    if (FILE* fp = std::fopen(cache, "r")) {
      long long v = 0;
      const int got = std::fscanf(fp, "max_batch=%lld", &v);
      std::fclose(fp);
      if (got == 1 && v >= 256 && v <= (1ll << 20)) return v;
    }
    *calibrate = true;
  }
  int64_t cap = 65536;
  if (ctx->budget) {
    const size_t room = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
    while (cap > 256 && (size_t)cap * m * sizeof(float) * 3 > room) cap /= 2;
  }
  return cap;
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
  bool calibrate = false;
  S->cap = pick_cap(own, basis, m, tune_cache, &calibrate);
  auto cleanup = [&](fkk_status e) {
    if (S->stream) cudaStreamDestroy(S->stream);
    if (e && own->last_error.size()) ctx->last_error = own->last_error;
    fkk_destroy(own);
    delete S;
    return e;
  };
  ctx = own;  // staging and calibration below use the server's context
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(ctx, FKK_ERR_CUDA, "fkk_serve_start: stream"));
  fkk_status s;
  char name[64];
  std::snprintf(name, sizeof name, "serve_in_%p", (void*)S);
  S->d_in = (float*)workspace(ctx, name, (size_t)S->cap * m * sizeof(float), &s);
  if (!S->d_in) return cleanup(s);
  std::snprintf(name, sizeof name, "serve_out_%p", (void*)S);
  S->d_out = (float*)workspace(ctx, name, (size_t)S->cap * m * sizeof(float), &s);
  if (!S->d_out) return cleanup(s);
  if (calibrate) {
    // time fkk_apply on ratio-one tiles of the staging size and below
    FKK_COUNT_LAUNCH();
    fill_kernel<<<(unsigned)(((int64_t)S->cap * m + 255) / 256), 256, 0, S->stream>>>(S->d_in, (int64_t)S->cap * m,
                                                                                       1.0f);
    double best = 0.0;
    std::vector<std::pair<int64_t, double>> rates;
    for (int64_t c = 2048; c <= S->cap; c *= 2) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      fkk_apply(ctx, basis, S->d_in, c, m, S->d_out, nullptr, m, S->stream);  // warm
      cudaEventRecord(e0, S->stream);
      for (int r = 0; r < 3; ++r) fkk_apply(ctx, basis, S->d_in, c, m, S->d_out, nullptr, m, S->stream);
      cudaEventRecord(e1, S->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      const double rate = 3.0 * (double)c / (ms > 0.f ? ms : 1e-3f);
      rates.emplace_back(c, rate);
      best = std::max(best, rate);
    }
    for (auto& r : rates)
      if (r.second >= 0.9 * best) {
        S->cap = r.first;
        break;
      }
    if (FILE* fp = std::fopen(tune_cache, "w")) {
      std::fprintf(fp, "max_batch=%lld\n", (long long)S->cap);
      std::fclose(fp);
    }
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return FKK_OK;
}

fkk_status fkk_serve_submit(fkk_server* S, const float* tile, int64_t n_spectra, int32_t tile_on_host,
                            float* im_out, fkk_req* out_id) {
  if (!S || !tile || !im_out || !out_id || n_spectra < 1) return FKK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) return FKK_ERR_SHUTDOWN;
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
  // tiles larger than the staging buffers run alone (a device tile in
  // place, a host tile in chunks); submission order is kept
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

fkk_status fkk_serve_stop(fkk_server* S) {
  if (!S) return FKK_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    // queued requests are cancelled; a batch already running completes
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
  cudaStreamDestroy(S->stream);
  fkk_destroy(S->ctx);  // staging buffers and all workspace of the server
  delete S;
  return FKK_OK;
}

}  // extern "C"
