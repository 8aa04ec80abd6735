// Reconstruction on the tensor cores, Eq. fKKEC with U S = P:
//   Im{K}[n, j] = exp((P C_amp)[n, j]) sin((P C_ph)[n, j]),  Re with cos.
//
// GEMM  D[n, 2j + t] = sum_i P[n, i] C_t[i, j]  (t = 0 amp, 1 phase), i.e.
// N x Kp times Kp x 2M with the amplitude and phase coefficient columns
// interleaved, so the accumulator row of spectrum n holds (amp, phase)
// pairs of consecutive channels and the epilogue needs no exchange.
// Operands are bf16 hi + lo (three products, fp32 accumulation), K-major
// with the 128-byte swizzle, Kp = 64 or 128 (k zero-padded).
//
// Persistent CTAs: warp 0 issues TMA (the 128-spectrum A tile once per row
// tile, 256-column B tiles through a 2-stage ring), warp 1 issues
// tcgen05.mma into two 256-column TMEM accumulators, 8 or 16 warps after them read
// the accumulators (one TMEM lane per spectrum), evaluate exp / sin / cos
// with the fast intrinsics, and store the outputs: each 32-spectrum x
// 32-channel block goes into a 128-byte-swizzled staging tile that one TMA
// store writes (clipping rows and channels outside the arrays), or, when the
// output rows are not 16-byte aligned, through a transpose buffer as
// coalesced row stores.  The epilogue of one column tile overlaps the MMAs
// of the next.
#include "common.cuh"
#include "fit.h"
#include "tc.cuh"

namespace fkk {
namespace {

constexpr int kTM = 128, kTN = 256;
constexpr int kMaxStages = 2;
// warp 0 TMA, warp 1 MMA, then 8 epilogue warps, or 16 for the TMA-store
// path without Re (its staging tiles fit shared memory twice over)
constexpr int kEpiWarpsRow = 8, kEpiWarpsTma = 16;
template <int kEpi>
constexpr int rec_threads() { return 64 + 32 * kEpi; }

struct ReconArgs {
  int64_t n;        // spectra
  int m;            // channels
  int kp;           // padded K (64 or 128)
  int n_row_tiles;  // ceil(n / 128)
  int n_col_tiles;  // ceil(2m / 256)
  int nst;          // B ring depth (2 for Kp = 64, 1 for Kp = 128)
  float* im;
  float* re;
  int64_t ld_out;
  long long* status;
  const float* bias;  // linear mode: added to channel j of every row (may be null)
};

__device__ __forceinline__ uint32_t a_bytes(int kp) { return kTM * kp * 2; }
__device__ __forceinline__ uint32_t b_bytes(int kp) { return kTN * kp * 2; }

// 16-byte chunk q of row r of a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128(int r, int q) { return (uint32_t)(r * 128 + ((q ^ (r & 7)) << 4)); }

// kLinear: the output is the amplitude accumulator itself plus a per-channel
// bias (P C + 1 b^T), with no exp / sin and no Re output.  kTma: outputs
// leave through TMA stores (tm_im, tm_re) instead of per-row stores.  kEpi:
// epilogue warps, four per TMEM lane quarter share a tile's columns.
template <bool kLinear, bool kTma, int kEpiWarps>
__global__ void __launch_bounds__(rec_threads<kEpiWarps>(), 1)
    recon_tc_kernel(const __grid_constant__ CUtensorMap tp_hi, const __grid_constant__ CUtensorMap tp_lo,
                    const __grid_constant__ CUtensorMap tc_hi, const __grid_constant__ CUtensorMap tc_lo,
                    const __grid_constant__ CUtensorMap tm_im, const __grid_constant__ CUtensorMap tm_re,
                    ReconArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kp = p.kp;
  const int kch = kp / 64;  // 64-wide K chunks (128-byte swizzled rows)
  // layout: A_hi | A_lo | stages x (B_hi | B_lo) | barriers
  uint8_t* a_hi = smem;
  uint8_t* a_lo = a_hi + a_bytes(kp);
  uint8_t* bstage = a_lo + a_bytes(kp);
  const uint32_t bst = 2 * b_bytes(kp);
  // TMA output staging (1024-aligned): per epilogue warp a 32 x 32 fp32 tile for Im (and one for Re)
  uint8_t* ostage = bstage + p.nst * bst;
  const uint32_t ostg_warp = (p.re ? 2 : 1) * 4096;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ostage + (kTma ? kEpiWarps * ostg_warp : 0));
  uint64_t* a_full = bars;                 // A tile loaded
  uint64_t* a_empty = bars + 1;            // A tile consumed (all MMAs of the row tile done)
  uint64_t* b_full = bars + 2;             // [kMaxStages]
  uint64_t* b_empty = b_full + kMaxStages; // [kMaxStages]
  uint64_t* acc_full = b_empty + kMaxStages;   // [2] accumulator ready for the epilogue
  uint64_t* acc_empty = acc_full + 2;          // [2] accumulator drained (4 epilogue warps arrive)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  // row-store path: per epilogue warp a 32 x 33 transpose block
  float* xpose = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + 256);
  __shared__ int fail_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    fail_s = 0;
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, 1);
    for (int s = 0; s < kMaxStages; ++s) {
      tc::mbar_init(&b_full[s], 1);
      tc::mbar_init(&b_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&acc_full[s], 1);
      tc::mbar_init(&acc_empty[s], kEpiWarps);
    }
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tp_hi);
    tc::prefetch_tmap(&tp_lo);
    tc::prefetch_tmap(&tc_hi);
    tc::prefetch_tmap(&tc_lo);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const uint32_t ab = a_bytes(kp), bb = b_bytes(kp);

  if (warp == 0 && lane == 0) {
    // ---------------- producer ----------------
    int it = 0;       // B tile counter (ring position)
    int rt_local = 0; // row tiles handled by this CTA
    for (int rt = blockIdx.x; rt < p.n_row_tiles; rt += gridDim.x, ++rt_local) {
      if (!tc::mbar_wait(a_empty, (rt_local & 1) ^ 1)) { fail_s = 1; break; }
      tc::mbar_arrive_expect_tx(a_full, 2 * ab);
      for (int c = 0; c < kch; ++c) {
        tc::tma_load_2d(a_hi + c * (kTM * 128), &tp_hi, a_full, c * 64, rt * kTM);
        tc::tma_load_2d(a_lo + c * (kTM * 128), &tp_lo, a_full, c * 64, rt * kTM);
      }
      for (int ct = 0; ct < p.n_col_tiles; ++ct, ++it) {
        const int s = it % p.nst;
        const uint32_t ph = (it / p.nst) & 1;
        if (!tc::mbar_wait(&b_empty[s], ph ^ 1)) { fail_s = 1; break; }
        uint8_t* bh = bstage + s * bst;
        uint8_t* bl = bh + bb;
        tc::mbar_arrive_expect_tx(&b_full[s], 2 * bb);
        for (int c = 0; c < kch; ++c) {
          tc::tma_load_2d(bh + c * (kTN * 128), &tc_hi, &b_full[s], c * 64, ct * kTN);
          tc::tma_load_2d(bl + c * (kTN * 128), &tc_lo, &b_full[s], c * 64, ct * kTN);
        }
      }
      if (fail_s) break;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, kTN);
    int it = 0, rt_local = 0, acc_it = 0;
    for (int rt = blockIdx.x; rt < p.n_row_tiles; rt += gridDim.x, ++rt_local) {
      if (!tc::mbar_wait(a_full, rt_local & 1)) { fail_s = 1; break; }
      tc::tc_fence_after();
      for (int ct = 0; ct < p.n_col_tiles; ++ct, ++it, ++acc_it) {
        const int s = it % p.nst;
        const uint32_t ph = (it / p.nst) & 1;
        const int acc = acc_it & 1;
        const uint32_t aph = (acc_it >> 1) & 1;
        if (!tc::mbar_wait(&acc_empty[acc], aph ^ 1)) { fail_s = 1; break; }
        if (!tc::mbar_wait(&b_full[s], ph)) { fail_s = 1; break; }
        tc::tc_fence_after();
        const uint32_t d = tbase + acc * kTN;
        const uint32_t ah = tc::smem_u32(a_hi), al = tc::smem_u32(a_lo);
        const uint32_t bh = tc::smem_u32(bstage + s * bst), bl = bh + bb;
        bool first = true;
        for (int c = 0; c < kch; ++c) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t ao = c * (kTM * 128) + kk * 32, bo = c * (kTN * 128) + kk * 32;
            tc::mma_bf16(d, tc::sdesc_kmajor_sw128(ah + ao), tc::sdesc_kmajor_sw128(bh + bo), idesc, first ? 0u : 1u);
            tc::mma_bf16(d, tc::sdesc_kmajor_sw128(ah + ao), tc::sdesc_kmajor_sw128(bl + bo), idesc, 1u);
            tc::mma_bf16(d, tc::sdesc_kmajor_sw128(al + ao), tc::sdesc_kmajor_sw128(bh + bo), idesc, 1u);
            first = false;
          }
        }
        tc::mma_commit(&b_empty[s]);
        tc::mma_commit(&acc_full[acc]);
      }
      if (fail_s) break;
      tc::mma_commit(a_empty);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    // warps 2..9: TMEM lane quarter q = warp % 4 (the rule for tcgen05.ld),
    // column half h of each 256-column tile
    const int ew = warp - 2;
    const int q = warp & 3;
    const int h = ew >> 2;
    float* tbuf = xpose + ew * (32 * 33);
    int acc_it = 0;
    for (int rt = blockIdx.x; rt < p.n_row_tiles; rt += gridDim.x) {
      const int64_t n0 = (int64_t)rt * kTM + q * 32;
      const int64_t left = p.n - n0;
      const int rows = left < 32 ? (int)(left > 0 ? left : 0) : 32;
      for (int ct = 0; ct < p.n_col_tiles; ++ct, ++acc_it) {
        const int acc = acc_it & 1;
        const uint32_t aph = (acc_it >> 1) & 1;
        if (!tc::mbar_wait(&acc_full[acc], aph)) { fail_s = 1; break; }
        tc::tc_fence_after();
        const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + acc * kTN;
        // two TMEM loads (32 channel pairs) -> a 32 x 32 output block in shared
        // memory (row = spectrum) -> stores of 32 consecutive channels per row
#pragma unroll 1
        constexpr int kBlk = (kTN / 64) / (kEpiWarps / 4);  // 32-channel blocks per warp and tile
        for (int c64 = h * kBlk; c64 < (h + 1) * kBlk && kTma; ++c64) {
          uint8_t* so = ostage + ew * ostg_warp;
          const bool with_re = kEpiWarps == kEpiWarpsRow && p.re != nullptr;  // the wide form writes Im only
          float im32[32], re32[32];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            float v[32];
            tc::tmem_ld32(taddr + c64 * 64 + hh * 32, v);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const float ea = __expf(v[2 * t]);
              if (with_re) {
                float sn, cn;
                __sincosf(v[2 * t + 1], &sn, &cn);
                im32[hh * 16 + t] = ea * sn;
                re32[hh * 16 + t] = ea * cn;
              } else {
                im32[hh * 16 + t] = ea * __sinf(v[2 * t + 1]);
              }
            }
          }
          if (lane == 0) tc::bulk_wait_read0();  // the previous stores have read the staging tile(s)
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            *reinterpret_cast<float4*>(so + sw128(lane, q)) =
                make_float4(im32[4 * q], im32[4 * q + 1], im32[4 * q + 2], im32[4 * q + 3]);
            if (with_re)
              *reinterpret_cast<float4*>(so + 4096 + sw128(lane, q)) =
                  make_float4(re32[4 * q], re32[4 * q + 1], re32[4 * q + 2], re32[4 * q + 3]);
          }
          tc::fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            const int j0 = ct * (kTN / 2) + c64 * 32;
            tc::tma_store_2d(&tm_im, so, j0, (int)n0);
            if (with_re) tc::tma_store_2d(&tm_re, so + 4096, j0, (int)n0);
            tc::bulk_commit();
          }
        }
#pragma unroll 1
        for (int c64 = h * kBlk; c64 < (h + 1) * kBlk && !kTma; ++c64) {
          float ex[32], cs[32];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            float v[32];
            tc::tmem_ld32(taddr + c64 * 64 + hh * 32, v);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              if (kLinear) {
                tbuf[lane * 33 + hh * 16 + t] = v[2 * t];
              } else {
                float sn;
                __sincosf(v[2 * t + 1], &sn, &cs[hh * 16 + t]);
                ex[hh * 16 + t] = __expf(v[2 * t]);
                tbuf[lane * 33 + hh * 16 + t] = ex[hh * 16 + t] * sn;
              }
            }
          }
          __syncwarp();
          const int j = ct * (kTN / 2) + c64 * 32 + lane;  // this lane's channel
          if (j < p.m) {
            const float bj = (kLinear && p.bias) ? p.bias[j] : 0.f;
            for (int r = 0; r < rows; ++r) p.im[(n0 + r) * p.ld_out + j] = tbuf[r * 33 + lane] + bj;
          }
          __syncwarp();
          if (!kLinear && p.re) {
#pragma unroll
            for (int t = 0; t < 32; ++t) tbuf[lane * 33 + t] = ex[t] * cs[t];
            __syncwarp();
            if (j < p.m)
              for (int r = 0; r < rows; ++r) p.re[(n0 + r) * p.ld_out + j] = tbuf[r * 33 + lane];
            __syncwarp();
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
      }
      if (fail_s) break;
    }
  }
  if (kTma && warp >= 2 && lane == 0) tc::bulk_wait0();  // this warp's stores are complete
  __syncthreads();
  if (fail_s && threadIdx.x == 0) record_error(p.status, kErrTimeout);
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

// P (n x k fp32) -> hi / lo bf16 (n_pad x kp, zero padded).  One thread per
// 8 columns of a row (kp / 8 = 1 << g_shift groups per row): 16-byte stores
// of each term.
__global__ void pack_p_kernel(const float* __restrict__ p, int64_t n, int k, int64_t n_pad, int kp, int g_shift,
                              __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (n_pad * kp) >> 3) return;
  const int64_t r = t >> g_shift;
  const int c0 = (int)(t - (r << g_shift)) * 8;
  float v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = (r < n && c0 + q < k) ? p[r * k + c0 + q] : 0.f;
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
    h[q] = *reinterpret_cast<const uint32_t*>(&hb);
    l[q] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  *reinterpret_cast<uint4*>(hi + r * kp + c0) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + r * kp + c0) = make_uint4(l[0], l[1], l[2], l[3]);
}

// C (k x m fp64 amp and phase) -> interleaved rows (2m_pad x kp): row 2j = amp
// column j, row 2j + 1 = phase column j.
__global__ void pack_c_kernel(const double* __restrict__ camp, const double* __restrict__ cph, int k, int m,
                              int rows_pad, int kp, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows_pad * kp) return;
  const int r = (int)(t / kp), c = (int)(t % kp);
  const int j = r >> 1;
  float v = 0.f;
  if (j < m && c < k) v = (float)((r & 1) ? cph[(int64_t)c * m + j] : camp[(int64_t)c * m + j]);
  __nv_bfloat16 h, l;
  split_bf16(v, h, l);
  hi[t] = h;
  lo[t] = l;
}

size_t recon_smem(int kp, int nst, bool tma, bool re) {
  // TMA staging tiles, or the transpose buffers of the row-store path
  const size_t epi = tma ? (re ? (size_t)kEpiWarpsRow * 2 * 4096 : (size_t)kEpiWarpsTma * 4096)
                         : (size_t)kEpiWarpsRow * 32 * 33 * sizeof(float);
  return 1024 + 2 * (size_t)kTM * kp * 2 + (size_t)nst * 2 * kTN * kp * 2 + 256 + epi;
}

// Packs P and C into the given scratch and launches the kernel.
fkk_status recon_tc_run(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                        const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st, void* p_hi,
                        void* p_lo, void* c_hi, void* c_lo, bool linear, const float* bias) {
  const int kp = k <= 64 ? 64 : 128;
  const int64_t n_pad = ((n + kTM - 1) / kTM) * kTM;
  const int rows_c = ((2 * m + kTN - 1) / kTN) * kTN;
  __nv_bfloat16* phi = static_cast<__nv_bfloat16*>(p_hi);
  __nv_bfloat16* plo = static_cast<__nv_bfloat16*>(p_lo);
  __nv_bfloat16* chi = static_cast<__nv_bfloat16*>(c_hi);
  __nv_bfloat16* clo = static_cast<__nv_bfloat16*>(c_lo);
  {
    const int64_t tot = (n_pad * kp) >> 3;  // 8 columns per thread
    FKK_COUNT_LAUNCH();
    pack_p_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(p, n, k, n_pad, kp, kp == 64 ? 3 : 4, phi, plo);
    const int64_t totc = (int64_t)rows_c * kp;
    FKK_COUNT_LAUNCH();
    pack_c_kernel<<<(unsigned)((totc + 255) / 256), 256, 0, st>>>(c_amp, c_ph, k, m, rows_c, kp, chi, clo);
    FKK_CUDA(ctx, cudaGetLastError());
  }
  CUtensorMap tph, tpl, tch, tcl;
  const uint64_t rb = (uint64_t)kp * 2;
  FKK_TRY(make_tmap_2d(ctx, &tph, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, phi, kp, n_pad, rb, 64, kTM, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tpl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, plo, kp, n_pad, rb, 64, kTM, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tch, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, chi, kp, rows_c, rb, 64, kTN, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tcl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, clo, kp, rows_c, rb, 64, kTN, CU_TENSOR_MAP_SWIZZLE_128B));
  // TMA stores need 16-byte aligned output rows that also end on a 16-byte
  // boundary (a store clipped at the last channel still writes the rest of
  // its 16-byte granule, which would reach into a padded row's stride); the
  // staging must fit beside a 2-stage ring
  const bool want_re = !linear && re;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const bool tma = !linear && ld_out % 4 == 0 && m % 4 == 0 && al16(im) && (!want_re || al16(re)) &&
                   recon_smem(kp, 2, true, want_re) <= 227 * 1024;
  int nst = 2;
  if (recon_smem(kp, nst, tma, want_re) > 227 * 1024) nst = 1;
  const size_t smem = recon_smem(kp, nst, tma, want_re);
  if (smem > 227 * 1024) return fail(ctx, FKK_ERR_INVALID_ARG, "reconstruction tile does not fit shared memory");
  CUtensorMap tim, tre;
  if (tma) {
    FKK_TRY(make_tmap_2d(ctx, &tim, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, im, (uint64_t)m, (uint64_t)n,
                         (uint64_t)ld_out * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B));
    FKK_TRY(make_tmap_2d(ctx, &tre, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, want_re ? re : im, (uint64_t)m, (uint64_t)n,
                         (uint64_t)ld_out * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B));
  } else {
    tim = tph;  // unused by the kernel
    tre = tph;
  }
  const bool wide = tma && !want_re;  // 16 epilogue warps
  const void* fn = linear ? (const void*)recon_tc_kernel<true, false, kEpiWarpsRow>
                          : (tma ? (wide ? (const void*)recon_tc_kernel<false, true, kEpiWarpsTma>
                                         : (const void*)recon_tc_kernel<false, true, kEpiWarpsRow>)
                                 : (const void*)recon_tc_kernel<false, false, kEpiWarpsRow>);
  FKK_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ReconArgs a{n,      m,
              kp,     (int)(n_pad / kTM),
              rows_c / kTN, nst,
              im,     linear ? nullptr : re,
              ld_out, ctx->d_status,
              linear ? bias : nullptr};
  const int grid = (int)std::min<int64_t>(ctx->sm_count, a.n_row_tiles);
  FKK_COUNT_LAUNCH();
  if (linear)
    recon_tc_kernel<true, false, kEpiWarpsRow>
        <<<grid, rec_threads<kEpiWarpsRow>(), smem, st>>>(tph, tpl, tch, tcl, tim, tre, a);
  else if (wide)
    recon_tc_kernel<false, true, kEpiWarpsTma>
        <<<grid, rec_threads<kEpiWarpsTma>(), smem, st>>>(tph, tpl, tch, tcl, tim, tre, a);
  else if (tma)
    recon_tc_kernel<false, true, kEpiWarpsRow>
        <<<grid, rec_threads<kEpiWarpsRow>(), smem, st>>>(tph, tpl, tch, tcl, tim, tre, a);
  else
    recon_tc_kernel<false, false, kEpiWarpsRow>
        <<<grid, rec_threads<kEpiWarpsRow>(), smem, st>>>(tph, tpl, tch, tcl, tim, tre, a);
  return cuda_check(ctx, cudaGetLastError(), "recon_tc launch");
}

// The packed operands in the context's workspace.
fkk_status recon_tc_ws(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                       const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st, bool linear,
                       const float* bias) {
  fkk_status s;
  if (k > 128) return fail(ctx, FKK_ERR_INVALID_ARG, "k > 128");
  const int kp = k <= 64 ? 64 : 128;
  const int64_t n_pad = ((n + kTM - 1) / kTM) * kTM;
  const int rows_c = ((2 * m + kTN - 1) / kTN) * kTN;
  void* phi = workspace(ctx, "rtc_phi", (size_t)n_pad * kp * 2, &s);
  if (!phi) return s;
  void* plo = workspace(ctx, "rtc_plo", (size_t)n_pad * kp * 2, &s);
  if (!plo) return s;
  void* chi = workspace(ctx, "rtc_chi", (size_t)rows_c * kp * 2, &s);
  if (!chi) return s;
  void* clo = workspace(ctx, "rtc_clo", (size_t)rows_c * kp * 2, &s);
  if (!clo) return s;
  return recon_tc_run(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, st, phi, plo, chi, clo, linear, bias);
}

}  // namespace

fkk_status launch_reconstruct_tc(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                                 const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st) {
  return recon_tc_ws(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, st, false, nullptr);
}

fkk_status launch_reconstruct(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                              const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st) {
  return recon_tc_ws(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, st, false, nullptr);
}

fkk_status launch_reconstruct_linear(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c,
                                     const float* bias, float* out, int64_t ld_out, cudaStream_t st) {
  return recon_tc_ws(ctx, p, n, k, m, c, c, out, nullptr, ld_out, st, true, bias);
}

fkk_status launch_reconstruct_tc_scratch(fkk_ctx* ctx, const float* p, int64_t n, int k, int m,
                                         const double* c_amp, const double* c_ph, float* im, float* re,
                                         int64_t ld_out, cudaStream_t st, void* p_hi, void* p_lo, void* c_hi,
                                         void* c_lo) {
  if (k > 128) return fail(ctx, FKK_ERR_INVALID_ARG, "k > 128");
  return recon_tc_run(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, st, p_hi, p_lo, c_hi, c_lo, false, nullptr);
}

}  // namespace fkk
