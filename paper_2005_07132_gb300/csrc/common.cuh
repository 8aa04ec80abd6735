// Small device helpers shared by the fit kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace fkk {

constexpr long long kErrTimeout = -4;       // FKK_ERR_TIMEOUT
constexpr long long kErrNotConverged = -5;  // FKK_ERR_NOT_CONVERGED

// Record the first device-side error in the context status block.
__device__ __forceinline__ void record_error(long long* status, long long code) {
  atomicCAS(reinterpret_cast<unsigned long long*>(status), 0ull, (unsigned long long)code);
}

// d = hi + lo + O(2^-17 |d|): two bf16 terms of a float.
__device__ __forceinline__ void split_bf16(float d, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(d);
  lo = __float2bfloat16_rn(d - __bfloat162float(hi));
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide barrier for a cooperative launch with a bounded spin: a
// monotonic arrival counter (release on arrive, acquire on poll).  All
// blocks call it the same number of times with their own `target`, which
// starts at 0.  Returns false (and records FKK_ERR_TIMEOUT) if the wait
// exceeded `limit` polls, or if another block already gave up (abort flag).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned nblocks, unsigned& target, int* abort_flag,
                                          long long* status, unsigned limit = (1u << 21)) {
  __shared__ int ok_s;
  target += nblocks;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_add_release_gpu(count, 1u);
    unsigned it = 0;
    while (ld_acquire_gpu(count) < target) {
      if ((++it & 255) == 0) {
        if (*(volatile int*)abort_flag) { ok = 0; break; }
        if (it > limit) {
          ok = 0;
          atomicExch(abort_flag, 1);
          record_error(status, kErrTimeout);
          break;
        }
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace fkk
