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

// Grid-wide barrier for a cooperative launch with a bounded spin.  All
// blocks must call it the same number of times.  `bar` points at two
// unsigned words {arrived, generation} zeroed before the launch.  Returns
// false (and records FKK_ERR_TIMEOUT) if the wait exceeded ~`limit`
// polls, or if another block already gave up (abort flag set).
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned nblocks, int* abort_flag,
                                          long long* status, unsigned limit = (1u << 22)) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = bar + 1;
    unsigned g = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (*(volatile int*)abort_flag) { ok = 0; break; }
        if (++it > limit) {
          ok = 0;
          atomicExch(abort_flag, 1);
          record_error(status, kErrTimeout);
          break;
        }
        if (it > 512) __nanosleep(32);
      }
    }
    __threadfence();
    if (*(volatile int*)abort_flag) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace fkk
