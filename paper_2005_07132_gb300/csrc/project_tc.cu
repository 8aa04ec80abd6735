// Projection of the spectra on the basis on the tensor cores (Sec. 2.2,
// U S = A V; the sub-sample rows of Eqs. q_max / q_min come from its
// columns):
//   P[n, i] = sum_j d[n, j] Wf[j, i] + o_i,  Wf = f W,  o = c^T Wf,
// d the shifted log ratio of the transformed cube (channel-major bf16 hi +
// lo, spectra contiguous), W the basis.
//
// GEMM M = 128 spectra per row tile, N = k rounded up to 16, K = channels in
// blocks of 64.  The cube tile is the MN-major A operand: two TMA boxes of
// 64 spectra x 64 channels with the 128-byte swizzle (8 KB apart along M);
// f W is split into bf16 hi + lo and stored K-major as the B operand.  Four
// products per K step (hi/lo x hi/lo) accumulate in fp32 in TMEM, so the
// result carries only the representation error of the two operands.
//
// Persistent CTAs of 6 warps: warp 0 issues TMA through a 4-stage ring,
// warp 1 issues tcgen05.mma into two TMEM accumulators, warps 2..5 read a
// finished accumulator (one TMEM lane per spectrum), add o, store P and
// reduce each column's maximum / minimum over the tile to the candidates
// that argext_reduce_kernel combines (ties to the lowest row).
#include "common.cuh"
#include "fit.h"
#include "tc.cuh"

namespace fkk {
namespace {

constexpr int kTM = 128;      // spectra per row tile
constexpr int kKB = 64;       // channels per K block
constexpr int kStages = 4;
constexpr int kThreads = 192;  // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr uint32_t kBox = 64 * 64 * 2;  // one 64-spectrum x 64-channel bf16 box
constexpr uint32_t kABytes = 2 * kBox;  // A operand (128 spectra) per term

struct ProjTcArgs {
  int64_t n;
  int k;
  int nkb;          // channel blocks
  int n_row_tiles;  // ceil(n / 128)
  const float* off;
  float* p;         // n x k
  float4* cand;     // [n_row_tiles][k] (max, argmax, min, argmin) or null
  long long* status;
};

__host__ __device__ constexpr uint32_t stage_bytes(int kp) { return 2 * kABytes + 2u * kp * 128u; }

template <int KP>
__global__ void __launch_bounds__(kThreads, 1)
    project_tc_kernel(const __grid_constant__ CUtensorMap td_hi, const __grid_constant__ CUtensorMap td_lo,
                      const __grid_constant__ CUtensorMap tw_hi, const __grid_constant__ CUtensorMap tw_lo,
                      ProjTcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t kStage = stage_bytes(KP);
  constexpr uint32_t kBBytes = KP * 128u;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint64_t* full = bars;                    // [kStages]
  uint64_t* empty = full + kStages;         // [kStages]
  uint64_t* acc_full = empty + kStages;     // [2]
  uint64_t* acc_empty = acc_full + 2;       // [2], 4 epilogue warps arrive
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  float* redv = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + 256);  // [4][KP][2]
  int* redi = reinterpret_cast<int*>(redv + 4 * KP * 2);                           // [4][KP][2]
  __shared__ int fail_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    fail_s = 0;
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&acc_full[s], 1);
      tc::mbar_init(&acc_empty[s], 4);
    }
    tc::fence_mbar_init();
    tc::prefetch_tmap(&td_hi);
    tc::prefetch_tmap(&td_lo);
    tc::prefetch_tmap(&tw_hi);
    tc::prefetch_tmap(&tw_lo);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 256);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer ----------------
    int it = 0;
    for (int rt = blockIdx.x; rt < p.n_row_tiles && !fail_s; rt += gridDim.x) {
      for (int kb = 0; kb < p.nkb; ++kb, ++it) {
        const int s = it % kStages;
        const uint32_t ph = (it / kStages) & 1;
        if (!tc::mbar_wait(&empty[s], ph ^ 1)) { fail_s = 1; break; }
        uint8_t* st = smem + s * kStage;
        tc::mbar_arrive_expect_tx(&full[s], kStage);
        const int n0 = rt * kTM, j0 = kb * kKB;
        tc::tma_load_2d(st, &td_hi, &full[s], n0, j0);
        tc::tma_load_2d(st + kBox, &td_hi, &full[s], n0 + 64, j0);
        tc::tma_load_2d(st + kABytes, &td_lo, &full[s], n0, j0);
        tc::tma_load_2d(st + kABytes + kBox, &td_lo, &full[s], n0 + 64, j0);
        tc::tma_load_2d(st + 2 * kABytes, &tw_hi, &full[s], j0, 0);
        tc::tma_load_2d(st + 2 * kABytes + kBBytes, &tw_lo, &full[s], j0, 0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, KP) | tc::kIdescAMnMajor;
    int it = 0, acc_it = 0;
    for (int rt = blockIdx.x; rt < p.n_row_tiles && !fail_s; rt += gridDim.x, ++acc_it) {
      const int acc = acc_it & 1;
      const uint32_t aph = (acc_it >> 1) & 1;
      if (!tc::mbar_wait(&acc_empty[acc], aph ^ 1)) { fail_s = 1; break; }
      tc::tc_fence_after();
      const uint32_t d = tbase + acc * 128;
      for (int kb = 0; kb < p.nkb; ++kb, ++it) {
        const int s = it % kStages;
        const uint32_t ph = (it / kStages) & 1;
        if (!tc::mbar_wait(&full[s], ph)) { fail_s = 1; break; }
        tc::tc_fence_after();
        const uint32_t ah = tc::smem_u32(smem + s * kStage), al = ah + kABytes;
        const uint32_t bh = ah + 2 * kABytes, bl = bh + kBBytes;
#pragma unroll
        for (int kk = 0; kk < kKB / 16; ++kk) {
          // A: 16 channels = two 8-row groups (2 x 1024 B) further along K;
          // B: 16 channels = 32 bytes further inside the 128-byte row
          const uint64_t a_hi = tc::sdesc_mnmajor_sw128(ah + kk * 2048, kBox, 1024);
          const uint64_t a_lo = tc::sdesc_mnmajor_sw128(al + kk * 2048, kBox, 1024);
          const uint64_t b_hi = tc::sdesc_kmajor_sw128(bh + kk * 32);
          const uint64_t b_lo = tc::sdesc_kmajor_sw128(bl + kk * 32);
          tc::mma_bf16(d, a_hi, b_hi, idesc, (kb | kk) ? 1u : 0u);
          tc::mma_bf16(d, a_hi, b_lo, idesc, 1u);
          tc::mma_bf16(d, a_lo, b_hi, idesc, 1u);
          tc::mma_bf16(d, a_lo, b_lo, idesc, 1u);
        }
        tc::mma_commit(&empty[s]);
      }
      if (fail_s) break;
      tc::mma_commit(&acc_full[acc]);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;  // TMEM lane quarter (tcgen05.ld rule: warp % 4)
    const int eg = threadIdx.x - 64;  // 0..127 within the epilogue group
    int acc_it = 0;
    for (int rt = blockIdx.x; rt < p.n_row_tiles; rt += gridDim.x, ++acc_it) {
      const int acc = acc_it & 1;
      const uint32_t aph = (acc_it >> 1) & 1;
      // after a failed wait every epilogue warp still walks the same tiles
      // and named barriers, without touching TMEM or writing P
      bool live = !fail_s && tc::mbar_wait(&acc_full[acc], aph);
      if (!live) fail_s = 1;
      live = __all_sync(0xffffffffu, live);
      float v[KP];
#pragma unroll
      for (int i = 0; i < KP; ++i) v[i] = 0.f;
      if (live) {
        tc::tc_fence_after();
#pragma unroll
        for (int c = 0; c < KP / 16; ++c)
          tc::tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + acc * 128 + c * 16, v + c * 16);
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
      }
      const int64_t n = (int64_t)rt * kTM + q * 32 + lane;
      const bool valid = live && n < p.n;
#pragma unroll
      for (int i = 0; i < KP; ++i) v[i] += i < p.k ? p.off[i] : 0.f;
      if (valid) {
        float* row = p.p + n * p.k;
        if ((p.k & 3) == 0) {
#pragma unroll
          for (int i = 0; i < KP; i += 4)
            if (i < p.k) *reinterpret_cast<float4*>(row + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < KP; ++i)
            if (i < p.k) row[i] = v[i];
        }
      }
      if (p.cand) {
        // per column: (max, argmax, min, argmin) over the tile, ties to the lowest row
#pragma unroll
        for (int i = 0; i < KP; ++i) {
          if (i >= p.k) continue;  // uniform across the warp
          float mx = valid ? v[i] : -INFINITY, mn = valid ? v[i] : INFINITY;
          int imx = valid ? (int)n : 0x7fffffff, imn = imx;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, mx, o);
            int oi = __shfl_xor_sync(0xffffffffu, imx, o);
            if (ov > mx || (ov == mx && oi < imx)) { mx = ov; imx = oi; }
            ov = __shfl_xor_sync(0xffffffffu, mn, o);
            oi = __shfl_xor_sync(0xffffffffu, imn, o);
            if (ov < mn || (ov == mn && oi < imn)) { mn = ov; imn = oi; }
          }
          if (lane == 0) {
            redv[(q * KP + i) * 2] = mx;
            redi[(q * KP + i) * 2] = imx;
            redv[(q * KP + i) * 2 + 1] = mn;
            redi[(q * KP + i) * 2 + 1] = imn;
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (eg < p.k) {
          const int i = eg;
          float mx = redv[i * 2], mn = redv[i * 2 + 1];
          int imx = redi[i * 2], imn = redi[i * 2 + 1];
          for (int w = 1; w < 4; ++w) {
            float ov = redv[(w * KP + i) * 2];
            int oi = redi[(w * KP + i) * 2];
            if (ov > mx || (ov == mx && oi < imx)) { mx = ov; imx = oi; }
            ov = redv[(w * KP + i) * 2 + 1];
            oi = redi[(w * KP + i) * 2 + 1];
            if (ov < mn || (ov == mn && oi < imn)) { mn = ov; imn = oi; }
          }
          p.cand[(int64_t)rt * p.k + i] = make_float4(mx, __int_as_float(imx), mn, __int_as_float(imn));
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    }
  }
  __syncthreads();
  if (fail_s && threadIdx.x == 0) record_error(p.status, kErrTimeout);
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, 256);
}

// f W split into bf16 hi + lo, stored K-major [kp][mg] (zero padded), and
// o = c^T (f W) in fp64.
__global__ void prep_wt_kernel(const double* __restrict__ w, const double* __restrict__ f,
                               const float* __restrict__ c, int m, int k, int mg, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, float* __restrict__ off) {
  const int i = blockIdx.x;  // row of the B operand (basis column), < kp
  double acc = 0.0;
  for (int j = threadIdx.x; j < mg; j += blockDim.x) {
    float v = 0.f;
    if (i < k && j < m) {
      const double x = w[(int64_t)j * k + i] * (f ? f[j] : 1.0);
      v = (float)x;
      if (c) acc += (double)c[j] * x;
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    hi[(int64_t)i * mg + j] = h;
    lo[(int64_t)i * mg + j] = l;
  }
  if (!off || i >= k) return;
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    off[i] = (float)s;
  }
}

size_t proj_smem(int kp) { return 1024 + (size_t)kStages * stage_bytes(kp) + 256 + (size_t)4 * kp * 2 * 8; }

template <int KP>
fkk_status run_proj(fkk_ctx* ctx, const CUtensorMap* maps, const ProjTcArgs& a, cudaStream_t st) {
  const size_t smem = proj_smem(KP);
  if (smem > 227 * 1024) return fail(ctx, FKK_ERR_INVALID_ARG, "projection tile does not fit shared memory");
  FKK_CUDA(ctx, cudaFuncSetAttribute(project_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>(ctx->sm_count, a.n_row_tiles);
  FKK_COUNT_LAUNCH();
  project_tc_kernel<KP><<<grid, kThreads, smem, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  return cuda_check(ctx, cudaGetLastError(), "project_tc launch");
}

}  // namespace

fkk_status launch_project_tc(fkk_ctx* ctx, const DtLayout& L, const double* w, const double* f, int k, float* p,
                             float4* cand, cudaStream_t st) {
  fkk_status s;
  if (k < 1 || k > 80) return fail(ctx, FKK_ERR_INVALID_ARG, "projection: k = %d outside [1, 80]", k);
  const int kp = ((k + 15) / 16) * 16;
  __nv_bfloat16* whi = (__nv_bfloat16*)workspace(ctx, "ptc_whi", (size_t)kp * L.mg * 2, &s);
  if (!whi) return s;
  __nv_bfloat16* wlo = (__nv_bfloat16*)workspace(ctx, "ptc_wlo", (size_t)kp * L.mg * 2, &s);
  if (!wlo) return s;
  float* off = (float*)workspace(ctx, "ptc_off", (size_t)kp * 4, &s);
  if (!off) return s;
  FKK_COUNT_LAUNCH();
  prep_wt_kernel<<<kp, 256, 0, st>>>(w, f, L.c, L.m, k, L.mg, whi, wlo, off);
  FKK_CUDA(ctx, cudaGetLastError());
  CUtensorMap maps[4];
  // cube: inner = spectra (np, contiguous), outer = channels (mg); 64 x 64 boxes
  FKK_TRY(make_tmap_2d(ctx, &maps[0], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_hi, L.np, L.mg, (uint64_t)L.np * 2, 64,
                       64, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &maps[1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_lo, L.np, L.mg, (uint64_t)L.np * 2, 64,
                       64, CU_TENSOR_MAP_SWIZZLE_128B));
  // f W: inner = channels (mg), outer = basis rows (kp); 64 x kp boxes
  FKK_TRY(make_tmap_2d(ctx, &maps[2], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, whi, L.mg, kp, (uint64_t)L.mg * 2, 64,
                       kp, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &maps[3], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, wlo, L.mg, kp, (uint64_t)L.mg * 2, 64,
                       kp, CU_TENSOR_MAP_SWIZZLE_128B));
  ProjTcArgs a{L.n, k, L.mg / kKB, (int)((L.n + kTM - 1) / kTM), off, p, cand, ctx->d_status};
  switch (kp) {
    case 16: return run_proj<16>(ctx, maps, a, st);
    case 32: return run_proj<32>(ctx, maps, a, st);
    case 48: return run_proj<48>(ctx, maps, a, st);
    case 64: return run_proj<64>(ctx, maps, a, st);
    default: return run_proj<80>(ctx, maps, a, st);
  }
}

}  // namespace fkk
